// k_profiles.cu -- k-mer profiles on the device ("Multiplicity vector building
// phase", Algorithm 1, and the inverted index the sum-min kernel walks).
//
// Steps (one launch each unless noted):
//   encode_mark   residue -> 0..19, rolling base-20 code of every window
//                 (Eq. (1): windows of exactly k letters), one bit per code in
//                 a bitmap over all 20^k codes; letters outside the alphabet
//                 raise PD_ERR_ALPHABET.
//   (scan)        popcount prefix of the bitmap words -> dense id of a code is
//                 its rank among the codes present (an injective f, ascending
//                 with the code, "Multiplicity vector building phase").
//   mv_build      per gene: ids of its windows, sorted, run-length encoded into
//                 (id, multiplicity) pairs (Eqs. (2)-(3)); one count per
//                 distinct id goes to a histogram (postings per id).
//   (scan)        posting offsets from the histogram.
//   post_fill     scatter every (gene, count) into its id's posting list.
//   post_sort     sort each posting list by gene (warp per short list, block
//                 per long list) so the layout is deterministic and a gene
//                 range can be found by binary search.
#include "pd_internal.cuh"

namespace pdg {
namespace {

constexpr int kEncThreads = 256;
constexpr int kMvThreads = 256;
constexpr int kMvLongThreads = 1024;
constexpr int kFillThreads = 256;
constexpr uint32_t kSortSmemCap = 8192;  // keys sorted in shared memory per block

// ------------------------------------------------------------ encode_mark
__global__ void __launch_bounds__(kEncThreads)
    k_encode_mark(const uint8_t* __restrict__ res, const int64_t* __restrict__ gene_ptr, uint32_t n_genes, int k,
                  unsigned long long* __restrict__ bitmap, DevErr* err) {
  __shared__ uint8_t lut[256];
  init_letter_table(lut);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_genes; g += warps) {
    const int64_t r0 = gene_ptr[g];
    const uint32_t len = (uint32_t)(gene_ptr[g + 1] - r0);
    const uint8_t* s = res + r0;
    for (uint32_t p = lane; p < len; p += 32) {
      if (lut[s[p]] >= kAlphabetSize) raise_error(err, PD_ERR_ALPHABET, (unsigned long long)(r0 + p));
    }
    for (uint32_t p = lane; p + (uint32_t)k <= len; p += 32) {
      unsigned long long code = 0;
      bool ok = true;
      for (int t = 0; t < k; ++t) {
        uint32_t c = lut[s[p + t]];
        ok &= c < (uint32_t)kAlphabetSize;
        code = code * (unsigned long long)kAlphabetSize + (c < (uint32_t)kAlphabetSize ? c : 0u);
      }
      if (ok) atomicOr(&bitmap[code >> 6], 1ull << (code & 63u));
    }
  }
}

// ------------------------------------------------------------ mv_build
__device__ __forceinline__ uint32_t code_rank(unsigned long long code, const unsigned long long* __restrict__ bitmap,
                                              const uint32_t* __restrict__ word_rank) {
  const unsigned long long w = bitmap[code >> 6];
  const unsigned long long below = (1ull << (code & 63u)) - 1ull;
  return word_rank[code >> 6] + (uint32_t)__popcll(w & below);
}

// Multiplicity vector of gene g, with `keys` (shared or global) holding at
// least next_pow2(La) words.  Called by every thread of the block.
__device__ __forceinline__ void mv_build_one(uint32_t g, uint32_t* keys, const uint8_t* __restrict__ lut,
                                             uint32_t* warp_tmp, const uint8_t* __restrict__ res,
                                             const int64_t* __restrict__ gene_ptr,
                                             const uint32_t* __restrict__ win_off, int k,
                                             const unsigned long long* __restrict__ bitmap,
                                             const uint32_t* __restrict__ word_rank, uint32_t* __restrict__ mv_id,
                                             uint16_t* __restrict__ mv_cnt, uint32_t* __restrict__ mv_len,
                                             uint32_t* __restrict__ hist) {
  const uint32_t off = win_off[g];
  const uint32_t La = win_off[g + 1] - off;
  const uint8_t* s = res + gene_ptr[g];
  const uint32_t n2 = next_pow2(La);
  for (uint32_t p = threadIdx.x; p < n2; p += blockDim.x) {
    uint32_t key = kEmpty;
    if (p < La) {
      unsigned long long code = 0;
      for (int t = 0; t < k; ++t) {
        uint32_t c = lut[s[p + t]];
        code = code * (unsigned long long)kAlphabetSize + (c < (uint32_t)kAlphabetSize ? c : 0u);
      }
      key = code_rank(code, bitmap, word_rank);
    }
    keys[p] = key;
  }
  __syncthreads();
  if (n2 > 1) block_bitonic_sort(keys, n2);
  // run-length encoding: each thread owns a contiguous segment of positions
  const uint32_t seg = (La + blockDim.x - 1) / blockDim.x;
  const uint32_t p0 = min(La, threadIdx.x * seg), p1 = min(La, p0 + seg);
  uint32_t heads = 0;
  for (uint32_t p = p0; p < p1; ++p) heads += (p == 0 || keys[p] != keys[p - 1]) ? 1u : 0u;
  uint32_t total;
  uint32_t idx = block_exclusive_scan(heads, warp_tmp, &total);
  for (uint32_t p = p0; p < p1; ++p) {
    if (p == 0 || keys[p] != keys[p - 1]) {
      const uint32_t id = keys[p];
      uint32_t q = p + 1;
      while (q < La && keys[q] == id) ++q;
      mv_id[off + idx] = id;
      mv_cnt[off + idx] = (uint16_t)(q - p);
      atomicAdd(&hist[id], 1u);
      ++idx;
    }
  }
  if (threadIdx.x == 0) mv_len[g] = total;
  __syncthreads();
}

__global__ void __launch_bounds__(kMvThreads)
    k_mv_build_smem(const uint8_t* __restrict__ res, const int64_t* __restrict__ gene_ptr,
                    const uint32_t* __restrict__ win_off, uint32_t n_genes, int k,
                    const unsigned long long* __restrict__ bitmap, const uint32_t* __restrict__ word_rank,
                    uint32_t* __restrict__ mv_id, uint16_t* __restrict__ mv_cnt, uint32_t* __restrict__ mv_len,
                    uint32_t* __restrict__ hist, uint32_t max_sort) {
  extern __shared__ uint32_t keys[];
  __shared__ uint8_t lut[256];
  __shared__ uint32_t warp_tmp[kMvThreads / 32 + 1];
  init_letter_table(lut);
  for (uint32_t g = blockIdx.x; g < n_genes; g += gridDim.x) {
    const uint32_t La = win_off[g + 1] - win_off[g];
    if (next_pow2(La) > max_sort) continue;  // long gene: other kernel
    mv_build_one(g, keys, lut, warp_tmp, res, gene_ptr, win_off, k, bitmap, word_rank, mv_id, mv_cnt, mv_len,
                 hist);
  }
}

__global__ void __launch_bounds__(kMvLongThreads)
    k_mv_build_long(const uint8_t* __restrict__ res, const int64_t* __restrict__ gene_ptr,
                    const uint32_t* __restrict__ win_off, int k, const unsigned long long* __restrict__ bitmap,
                    const uint32_t* __restrict__ word_rank, uint32_t* __restrict__ mv_id,
                    uint16_t* __restrict__ mv_cnt, uint32_t* __restrict__ mv_len, uint32_t* __restrict__ hist,
                    const uint32_t* __restrict__ long_genes, uint32_t n_long, uint32_t* scratch,
                    const uint32_t* __restrict__ scratch_off) {
  __shared__ uint8_t lut[256];
  __shared__ uint32_t warp_tmp[kMvLongThreads / 32 + 1];
  init_letter_table(lut);
  for (uint32_t x = blockIdx.x; x < n_long; x += gridDim.x) {
    mv_build_one(long_genes[x], scratch + scratch_off[x], lut, warp_tmp, res, gene_ptr, win_off, k, bitmap,
                 word_rank, mv_id, mv_cnt, mv_len, hist);
  }
}

// ------------------------------------------------------------ post_fill
__global__ void __launch_bounds__(kFillThreads)
    k_post_fill(const uint32_t* __restrict__ win_off, const uint32_t* __restrict__ mv_len,
                const uint32_t* __restrict__ mv_id, const uint16_t* __restrict__ mv_cnt, uint32_t n_genes,
                const uint32_t* __restrict__ post_ptr, uint32_t* __restrict__ fill, uint32_t* __restrict__ post,
                uint32_t cnt_bits, uint32_t cnt_cap) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_genes; g += warps) {
    const uint32_t off = win_off[g], n = mv_len[g];
    for (uint32_t e = lane; e < n; e += 32) {
      const uint32_t id = mv_id[off + e];
      const uint32_t c = mv_cnt[off + e];
      const uint32_t pos = post_ptr[id] + atomicSub(&fill[id], 1u) - 1u;
      post[pos] = (g << cnt_bits) | (c < cnt_cap ? c : cnt_cap);
    }
  }
}

// ------------------------------------------------------------ post_sort
__global__ void __launch_bounds__(256)
    k_post_sort_warp(const uint32_t* __restrict__ post_ptr, uint64_t n_lists, uint32_t* __restrict__ post,
                     uint32_t* __restrict__ queue, uint32_t* __restrict__ queue_len) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_lists; w += warps) {
    const uint32_t lo = post_ptr[w], len = post_ptr[w + 1] - lo;
    if (len <= 1) continue;
    if (len > 32) {
      if (lane == 0) queue[atomicAdd(queue_len, 1u)] = (uint32_t)w;
      continue;
    }
    uint32_t x = (lane < len) ? post[lo + lane] : kEmpty;
    x = warp_sort32(x);
    if (lane < len) post[lo + lane] = x;
  }
}

__global__ void __launch_bounds__(256)
    k_post_sort_block(const uint32_t* __restrict__ post_ptr, uint32_t* __restrict__ post,
                      const uint32_t* __restrict__ queue, const uint32_t* __restrict__ queue_len) {
  extern __shared__ uint32_t keys[];
  const uint32_t n_q = *queue_len;
  for (uint32_t x = blockIdx.x; x < n_q; x += gridDim.x) {
    const uint32_t w = queue[x];
    const uint32_t lo = post_ptr[w], len = post_ptr[w + 1] - lo;
    const uint32_t n2 = next_pow2(len);
    if (n2 > kSortSmemCap) continue;  // handled by the long-list kernel
    for (uint32_t p = threadIdx.x; p < n2; p += blockDim.x) keys[p] = (p < len) ? post[lo + p] : kEmpty;
    __syncthreads();
    block_bitonic_sort(keys, n2);
    for (uint32_t p = threadIdx.x; p < len; p += blockDim.x) post[lo + p] = keys[p];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024)
    k_post_sort_long(const uint32_t* __restrict__ post_ptr, uint32_t* __restrict__ post,
                     const uint32_t* __restrict__ queue, const uint32_t* __restrict__ queue_len,
                     uint32_t* scratch) {
  const uint32_t n_q = *queue_len;
  for (uint32_t x = 0; x < n_q; ++x) {  // one block walks the queue in order
    const uint32_t w = queue[x];
    const uint32_t lo = post_ptr[w], len = post_ptr[w + 1] - lo;
    const uint32_t n2 = next_pow2(len);
    if (n2 <= kSortSmemCap) continue;
    for (uint32_t p = threadIdx.x; p < n2; p += blockDim.x) scratch[p] = (p < len) ? post[lo + p] : kEmpty;
    __syncthreads();
    block_bitonic_sort(scratch, n2);
    for (uint32_t p = threadIdx.x; p < len; p += blockDim.x) post[lo + p] = scratch[p];
    __syncthreads();
  }
}

// ------------------------------------------------------------ small helpers
__global__ void k_max_u32(const uint32_t* __restrict__ a, uint64_t n, uint32_t* out) {
  uint32_t m = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    m = max(m, a[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31u) == 0) atomicMax(out, m);
}

__global__ void k_gene_genome(const int32_t* __restrict__ genome_ptr, uint32_t n_genomes,
                              uint16_t* __restrict__ gene_genome) {
  for (uint32_t i = blockIdx.x; i < n_genomes; i += gridDim.x)
    for (int32_t g = genome_ptr[i] + (int32_t)threadIdx.x; g < genome_ptr[i + 1]; g += blockDim.x)
      gene_genome[g] = (uint16_t)i;
}

__global__ void k_select_codes(const unsigned long long* __restrict__ bitmap, const uint32_t* __restrict__ word_rank,
                               uint64_t n_words, unsigned long long* __restrict__ code_of_id) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_words;
       i += (uint64_t)gridDim.x * blockDim.x) {
    unsigned long long w = bitmap[i];
    uint32_t id = word_rank[i];
    while (w) {
      const int bit = __ffsll((long long)w) - 1;
      code_of_id[id++] = i * 64ull + (unsigned long long)bit;
      w &= w - 1ull;
    }
  }
}

__global__ void k_export_mv(ProfilesView P, const unsigned long long* __restrict__ mv_ptr,
                            const unsigned long long* __restrict__ code_of_id, unsigned long long* __restrict__ codes,
                            uint32_t* __restrict__ counts) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < P.n_genes; g += warps) {
    const uint32_t off = P.win_off[g];
    const unsigned long long dst = mv_ptr[g];
    for (uint32_t e = lane; e < P.mv_len[g]; e += 32) {
      if (codes) codes[dst + e] = code_of_id[P.mv_id[off + e]];
      if (counts) counts[dst + e] = P.mv_cnt[off + e];
    }
  }
}

// Exact count of k-mer id in gene g (binary search in its multiplicity vector).
__device__ __forceinline__ uint32_t mv_count_of(const ProfilesView& P, uint32_t g, uint32_t id) {
  uint32_t lo = P.win_off[g], hi = lo + P.mv_len[g];
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (P.mv_id[mid] < id) lo = mid + 1; else hi = mid;
  }
  return (lo < P.win_off[g] + P.mv_len[g] && P.mv_id[lo] == id) ? P.mv_cnt[lo] : 0u;
}

__global__ void k_export_index(ProfilesView P, int32_t* __restrict__ genes, uint32_t* __restrict__ counts) {
  const uint32_t mask = (P.cnt_bits >= 32) ? 0xFFFFFFFFu : ((1u << P.cnt_bits) - 1u);
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < P.n_entries;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t p = P.post[e];
    const uint32_t g = p >> P.cnt_bits;
    uint32_t c = p & mask;
    if (c == P.cnt_cap) {  // saturated: exact count from the gene's vector
      uint64_t lo = 0, hi = P.n_distinct;  // id = last w with post_ptr[w] <= e
      while (hi - lo > 1) {
        uint64_t mid = (lo + hi) >> 1;
        if (P.post_ptr[mid] <= e) lo = mid; else hi = mid;
      }
      c = mv_count_of(P, g, (uint32_t)lo);
    }
    if (genes) genes[e] = (int32_t)g;
    if (counts) counts[e] = c;
  }
}

unsigned grid_for(uint64_t items, unsigned per_block, unsigned cap) {
  uint64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

}  // namespace

#define PD_LAUNCH(L, name, ...)                              \
  do {                                                       \
    cudaError_t e_ = launch_begin(L, name);                  \
    if (e_ != cudaSuccess) return e_;                        \
    __VA_ARGS__;                                             \
    e_ = launch_end(L, name);                                \
    if (e_ != cudaSuccess) return e_;                        \
  } while (0)

cudaError_t run_encode_mark(Launcher* L, const uint8_t* res, const int64_t* gene_ptr, uint32_t n_genes, int k,
                            unsigned long long* bitmap, DevErr* err, cudaStream_t s) {
  const unsigned grid = grid_for((uint64_t)n_genes * 32, kEncThreads, 152u * 16u);
  PD_LAUNCH(L, "encode_mark", k_encode_mark<<<grid, kEncThreads, 0, s>>>(res, gene_ptr, n_genes, k, bitmap, err));
  return cudaSuccess;
}

cudaError_t run_mv_build(Launcher* L, const uint8_t* res, const int64_t* gene_ptr, const uint32_t* win_off,
                         uint32_t n_genes, int k, const unsigned long long* bitmap, const uint32_t* word_rank,
                         uint32_t* mv_id, uint16_t* mv_cnt, uint32_t* mv_len, uint32_t* hist,
                         const uint32_t* long_genes, uint32_t n_long, uint32_t* long_scratch,
                         const uint32_t* long_scratch_off, uint32_t max_smem_sort, cudaStream_t s) {
  const size_t smem = (size_t)max_smem_sort * sizeof(uint32_t);
  cudaError_t ea = cudaFuncSetAttribute(k_mv_build_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (ea != cudaSuccess) return ea;
  const unsigned grid = grid_for(n_genes, 1, 152u * 64u);
  PD_LAUNCH(L, "mv_build",
            k_mv_build_smem<<<grid, kMvThreads, smem, s>>>(res, gene_ptr, win_off, n_genes, k, bitmap, word_rank,
                                                            mv_id, mv_cnt, mv_len, hist, max_smem_sort));
  if (n_long) {
    PD_LAUNCH(L, "mv_build_long",
              k_mv_build_long<<<grid_for(n_long, 1, 152u), kMvLongThreads, 0, s>>>(
                  res, gene_ptr, win_off, k, bitmap, word_rank, mv_id, mv_cnt, mv_len, hist, long_genes, n_long,
                  long_scratch, long_scratch_off));
  }
  return cudaSuccess;
}

cudaError_t run_post_fill(Launcher* L, const uint32_t* win_off, const uint32_t* mv_len, const uint32_t* mv_id,
                          const uint16_t* mv_cnt, uint32_t n_genes, const uint32_t* post_ptr, uint32_t* fill,
                          uint32_t* post, uint32_t cnt_bits, uint32_t cnt_cap, cudaStream_t s) {
  const unsigned grid = grid_for((uint64_t)n_genes * 32, kFillThreads, 152u * 16u);
  PD_LAUNCH(L, "post_fill",
            k_post_fill<<<grid, kFillThreads, 0, s>>>(win_off, mv_len, mv_id, mv_cnt, n_genes, post_ptr, fill, post,
                                                       cnt_bits, cnt_cap));
  return cudaSuccess;
}

cudaError_t run_post_sort(Launcher* L, const uint32_t* post_ptr, uint64_t n_lists, uint32_t* post, uint32_t* queue,
                          uint32_t* queue_len, uint32_t max_posting, uint32_t* long_scratch, cudaStream_t s) {
  PD_LAUNCH(L, "post_sort_warp",
            k_post_sort_warp<<<grid_for(n_lists * 32, 256, 152u * 16u), 256, 0, s>>>(post_ptr, n_lists, post, queue,
                                                                                      queue_len));
  if (max_posting > 32) {
    const size_t smem = (size_t)kSortSmemCap * sizeof(uint32_t);
    cudaError_t ea = cudaFuncSetAttribute(k_post_sort_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ea != cudaSuccess) return ea;
    PD_LAUNCH(L, "post_sort_block",
              k_post_sort_block<<<152u * 4u, 256, smem, s>>>(post_ptr, post, queue, queue_len));
  }
  if (next_pow2(max_posting) > kSortSmemCap) {
    PD_LAUNCH(L, "post_sort_long", k_post_sort_long<<<1, 1024, 0, s>>>(post_ptr, post, queue, queue_len, long_scratch));
  }
  return cudaSuccess;
}

cudaError_t run_max_u32(Launcher* L, const uint32_t* a, uint64_t n, uint32_t* out, cudaStream_t s) {
  PD_LAUNCH(L, "max_u32", k_max_u32<<<grid_for(n, 256, 152u * 8u), 256, 0, s>>>(a, n, out));
  return cudaSuccess;
}

cudaError_t run_gene_genome(Launcher* L, const int32_t* genome_ptr, uint32_t n_genomes, uint16_t* gene_genome,
                            cudaStream_t s) {
  PD_LAUNCH(L, "gene_genome",
            k_gene_genome<<<grid_for(n_genomes, 1, 152u * 8u), 256, 0, s>>>(genome_ptr, n_genomes, gene_genome));
  return cudaSuccess;
}

cudaError_t run_select_codes(Launcher* L, const unsigned long long* bitmap, const uint32_t* word_rank,
                             uint64_t n_words, unsigned long long* code_of_id, cudaStream_t s) {
  PD_LAUNCH(L, "select_codes",
            k_select_codes<<<grid_for(n_words, 256, 152u * 16u), 256, 0, s>>>(bitmap, word_rank, n_words,
                                                                               code_of_id));
  return cudaSuccess;
}

cudaError_t run_export_mv(Launcher* L, const ProfilesView& P, const unsigned long long* mv_ptr,
                          const unsigned long long* code_of_id, unsigned long long* codes, uint32_t* counts,
                          cudaStream_t s) {
  PD_LAUNCH(L, "export_mv",
            k_export_mv<<<grid_for((uint64_t)P.n_genes * 32, 256, 152u * 16u), 256, 0, s>>>(P, mv_ptr, code_of_id,
                                                                                             codes, counts));
  return cudaSuccess;
}

cudaError_t run_export_index(Launcher* L, const ProfilesView& P, int32_t* genes, uint32_t* counts, cudaStream_t s) {
  PD_LAUNCH(L, "export_index",
            k_export_index<<<grid_for(P.n_entries, 256, 152u * 16u), 256, 0, s>>>(P, genes, counts));
  return cudaSuccess;
}

}  // namespace pdg
