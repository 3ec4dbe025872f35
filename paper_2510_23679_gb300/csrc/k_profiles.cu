// k_profiles.cu -- k-mer profiles on the device ("Multiplicity vector building
// phase", Algorithm 1, and the inverted index the sum-min kernel walks).
//
// Steps (one launch each):
//   encode_mark    residue -> 0..19, base-20 code of every window (Eq. (1):
//                  windows of exactly k letters), one bit per code in a bitmap
//                  over all 20^k codes; letters outside the alphabet raise
//                  PD_ERR_ALPHABET.
//   (scan)         popcount prefix of the bitmap words: the dense id of a code
//                  is its rank among the codes present (an injective f that is
//                  ascending with the code, "Multiplicity vector building").
//   mv_build       per gene: ids of its windows, sorted in shared memory,
//                  run-length encoded into (id, multiplicity) pairs (Eqs.
//                  (2)-(3)); also a min-hash of the gene's ids.
//   bucket_count   the inverted index is the transpose of the multiplicity
//   (scan)         vectors.  It is built in two levels: ids are grouped into
//   bucket_scatter at most 24576 buckets of 2^s consecutive ids; every (id,
//   bucket_fine    gene, count) record is scattered into its bucket (per-block
//                  histograms in shared memory reserve contiguous runs), then
//                  one block per bucket counts the records per id, writes the
//                  id offsets, places the postings and sorts each list by gene.
//   mv_post        each multiplicity-vector entry gets its posting range, so
//                  the sum-min kernel reads list bounds from its own
//                  (coalesced) vector instead of the id offset table.
//   order          queries ordered by min-hash buckets: genes that share their
//                  minimum hashed k-mer (likely homologs) run together and
//                  share posting lists in L2.
#include "pd_internal.cuh"

namespace pdg {
namespace {

constexpr int kEncThreads = 256;
constexpr int kMvThreads = 256;
constexpr int kMvLongThreads = 1024;
constexpr int kBucketThreads = 512;
constexpr int kFineThreads = 256;

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

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
                                             uint16_t* __restrict__ mv_cnt, uint32_t* __restrict__ mv_n,
                                             uint32_t* __restrict__ minhash) {
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
  uint32_t mh = kEmpty;
  for (uint32_t p = p0; p < p1; ++p) {
    if (p == 0 || keys[p] != keys[p - 1]) {
      const uint32_t id = keys[p];
      uint32_t q = p + 1;
      while (q < La && keys[q] == id) ++q;
      mv_id[off + idx] = id;
      mv_cnt[off + idx] = (uint16_t)(q - p);
      mh = min(mh, mix32(id));
      ++idx;
    }
  }
  // block minimum of the hashed ids (warp_tmp is free again after the scan)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mh = min(mh, __shfl_xor_sync(0xffffffffu, mh, o));
  if (threadIdx.x == 0) warp_tmp[0] = kEmpty;
  __syncthreads();
  if ((threadIdx.x & 31u) == 0) atomicMin(&warp_tmp[0], mh);
  __syncthreads();
  if (threadIdx.x == 0) {
    mv_n[g] = total;
    minhash[g] = warp_tmp[0];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kMvThreads)
    k_mv_build_smem(const uint8_t* __restrict__ res, const int64_t* __restrict__ gene_ptr,
                    const uint32_t* __restrict__ win_off, uint32_t n_genes, int k,
                    const unsigned long long* __restrict__ bitmap, const uint32_t* __restrict__ word_rank,
                    uint32_t* __restrict__ mv_id, uint16_t* __restrict__ mv_cnt, uint32_t* __restrict__ mv_n,
                    uint32_t* __restrict__ minhash, uint32_t max_sort) {
  extern __shared__ uint32_t keys[];
  __shared__ uint8_t lut[256];
  __shared__ uint32_t warp_tmp[kMvThreads / 32 + 1];
  init_letter_table(lut);
  for (uint32_t g = blockIdx.x; g < n_genes; g += gridDim.x) {
    const uint32_t La = win_off[g + 1] - win_off[g];
    if (next_pow2(La) > max_sort) continue;  // long gene: other kernel
    mv_build_one(g, keys, lut, warp_tmp, res, gene_ptr, win_off, k, bitmap, word_rank, mv_id, mv_cnt, mv_n,
                 minhash);
  }
}

__global__ void __launch_bounds__(kMvLongThreads)
    k_mv_build_long(const uint8_t* __restrict__ res, const int64_t* __restrict__ gene_ptr,
                    const uint32_t* __restrict__ win_off, int k, const unsigned long long* __restrict__ bitmap,
                    const uint32_t* __restrict__ word_rank, uint32_t* __restrict__ mv_id,
                    uint16_t* __restrict__ mv_cnt, uint32_t* __restrict__ mv_n, uint32_t* __restrict__ minhash,
                    const uint32_t* __restrict__ long_genes, uint32_t n_long, uint32_t* scratch,
                    const uint32_t* __restrict__ scratch_off) {
  __shared__ uint8_t lut[256];
  __shared__ uint32_t warp_tmp[kMvLongThreads / 32 + 1];
  init_letter_table(lut);
  for (uint32_t x = blockIdx.x; x < n_long; x += gridDim.x) {
    mv_build_one(long_genes[x], scratch + scratch_off[x], lut, warp_tmp, res, gene_ptr, win_off, k, bitmap,
                 word_rank, mv_id, mv_cnt, mv_n, minhash);
  }
}

// ------------------------------------------------------------ bucketed transpose
// Genes [g0, g1) of block b: a contiguous share of all genes.
__device__ __forceinline__ void block_gene_range(uint32_t n_genes, uint32_t* g0, uint32_t* g1) {
  const uint64_t per = ((uint64_t)n_genes + gridDim.x - 1) / gridDim.x;
  *g0 = (uint32_t)(per * blockIdx.x < n_genes ? per * blockIdx.x : n_genes);
  *g1 = (uint32_t)(per * (blockIdx.x + 1) < n_genes ? per * (blockIdx.x + 1) : n_genes);
}

__global__ void __launch_bounds__(kBucketThreads)
    k_bucket_count(const uint32_t* __restrict__ win_off, const uint32_t* __restrict__ mv_n,
                   const uint32_t* __restrict__ mv_id, uint32_t n_genes, uint32_t shift, uint32_t n_buckets,
                   uint32_t* __restrict__ bucket_count) {
  extern __shared__ uint32_t hist[];
  for (uint32_t b = threadIdx.x; b < n_buckets; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  uint32_t g0, g1;
  block_gene_range(n_genes, &g0, &g1);
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
  for (uint32_t g = g0 + warp; g < g1; g += n_warps) {
    const uint32_t off = win_off[g], n = mv_n[g];
    for (uint32_t e = lane; e < n; e += 32) atomicAdd(&hist[mv_id[off + e] >> shift], 1u);
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < n_buckets; b += blockDim.x)
    if (hist[b]) atomicAdd(&bucket_count[b], hist[b]);
}

__global__ void __launch_bounds__(kBucketThreads)
    k_bucket_scatter(const uint32_t* __restrict__ win_off, const uint32_t* __restrict__ mv_n,
                     const uint32_t* __restrict__ mv_id, const uint16_t* __restrict__ mv_cnt, uint32_t n_genes,
                     uint32_t shift, uint32_t n_buckets, uint32_t* __restrict__ bucket_cursor, uint32_t cnt_bits,
                     uint32_t cnt_cap, unsigned long long* __restrict__ recs) {
  extern __shared__ uint32_t hist[];  // n_buckets counts, then n_buckets bases
  uint32_t* base = hist + n_buckets;
  for (uint32_t b = threadIdx.x; b < n_buckets; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  uint32_t g0, g1;
  block_gene_range(n_genes, &g0, &g1);
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
  for (uint32_t g = g0 + warp; g < g1; g += n_warps) {
    const uint32_t off = win_off[g], n = mv_n[g];
    for (uint32_t e = lane; e < n; e += 32) atomicAdd(&hist[mv_id[off + e] >> shift], 1u);
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < n_buckets; b += blockDim.x)
    base[b] = hist[b] ? atomicAdd(&bucket_cursor[b], hist[b]) : 0u;
  __syncthreads();
  for (uint32_t g = g0 + warp; g < g1; g += n_warps) {
    const uint32_t off = win_off[g], n = mv_n[g];
    for (uint32_t e = lane; e < n; e += 32) {
      const uint32_t id = mv_id[off + e];
      const uint32_t c = mv_cnt[off + e];
      const uint32_t pos = atomicAdd(&base[id >> shift], 1u);
      recs[pos] = ((unsigned long long)id << 32) | (g << cnt_bits) | (c < cnt_cap ? c : cnt_cap);
    }
  }
}

// One block per bucket: counting sort of the bucket's records by id, then
// each id's postings sorted by gene (gene ids are unique within a list).
__global__ void __launch_bounds__(kFineThreads)
    k_bucket_fine(const uint32_t* __restrict__ bucket_start, uint32_t n_buckets, uint32_t shift, uint64_t n_ids_total,
                  unsigned long long* __restrict__ recs, uint32_t* __restrict__ post_ptr, uint32_t* __restrict__ post,
                  uint32_t* __restrict__ max_posting) {
  extern __shared__ uint32_t cnt[];  // 2^shift counters, then the long-list queue
  __shared__ uint32_t warp_tmp[kFineThreads / 32 + 1];
  __shared__ uint32_t n_long;
  const uint32_t ids_per = 1u << shift;
  uint32_t* longq = cnt + ids_per;
  const uint32_t items = (ids_per + kFineThreads - 1) / kFineThreads;
  uint32_t my_max = 0;
  for (uint32_t bk = blockIdx.x; bk < n_buckets; bk += gridDim.x) {
    const uint64_t id0 = (uint64_t)bk << shift;
    const uint32_t n_ids = (uint32_t)(n_ids_total - id0 < ids_per ? n_ids_total - id0 : ids_per);
    const uint32_t r0 = bucket_start[bk], R = bucket_start[bk + 1] - r0;
    for (uint32_t i = threadIdx.x; i < ids_per; i += kFineThreads) cnt[i] = 0;
    if (threadIdx.x == 0) n_long = 0;
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < R; r += kFineThreads)
      atomicAdd(&cnt[(uint32_t)(recs[r0 + r] >> 32) - (uint32_t)id0], 1u);
    __syncthreads();
    // exclusive scan of the per-id counts (each thread owns `items` consecutive ids)
    uint32_t sum = 0;
    for (uint32_t t = 0; t < items; ++t) {
      const uint32_t i = threadIdx.x * items + t;
      if (i < ids_per) sum += cnt[i];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan(sum, warp_tmp, &tot);
    for (uint32_t t = 0; t < items; ++t) {
      const uint32_t i = threadIdx.x * items + t;
      if (i < ids_per) {
        const uint32_t c = cnt[i];
        cnt[i] = run;  // becomes the placement cursor
        if (i < n_ids) post_ptr[id0 + i] = r0 + run;
        my_max = max(my_max, c);
        run += c;
      }
    }
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < R; r += kFineThreads) {
      const unsigned long long v = recs[r0 + r];
      const uint32_t pos = atomicAdd(&cnt[(uint32_t)(v >> 32) - (uint32_t)id0], 1u);
      post[r0 + pos] = (uint32_t)v;
    }
    __syncthreads();
    // cnt[i] now holds the end of list i; list i starts at cnt[i-1] (or 0).
    for (uint32_t i = threadIdx.x; i < n_ids; i += kFineThreads) {
      const uint32_t lo = i ? cnt[i - 1] : 0u, hi = cnt[i], len = hi - lo;
      if (len <= 1) continue;
      if (len > 24) {
        longq[atomicAdd(&n_long, 1u)] = i;
        continue;
      }
      uint32_t* L = post + r0 + lo;  // insertion sort in place (L1-resident)
      for (uint32_t x = 1; x < len; ++x) {
        const uint32_t v = L[x];
        uint32_t y = x;
        while (y > 0 && L[y - 1] > v) {
          L[y] = L[y - 1];
          --y;
        }
        L[y] = v;
      }
    }
    __syncthreads();
    // longer lists: one warp each, rank placement through the dead record area
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (uint32_t q = warp; q < n_long; q += kFineThreads / 32) {
      const uint32_t i = longq[q];
      const uint32_t lo = i ? cnt[i - 1] : 0u, len = cnt[i] - lo;
      uint32_t* L = post + r0 + lo;
      uint32_t* tmp = (uint32_t*)(recs + r0) + lo;  // disjoint per list
      for (uint32_t x = lane; x < len; x += 32) {
        const uint32_t v = L[x];
        uint32_t rank = 0;
        for (uint32_t y = 0; y < len; ++y) rank += (L[y] < v) ? 1u : 0u;
        tmp[rank] = v;
      }
      __syncwarp();
      for (uint32_t x = lane; x < len; x += 32) L[x] = tmp[x];
      __syncwarp();
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_max = max(my_max, __shfl_xor_sync(0xffffffffu, my_max, o));
  if ((threadIdx.x & 31u) == 0) atomicMax(max_posting, my_max);
}

// Every multiplicity-vector entry gets its posting range [mv_post, +mv_plen).
__global__ void __launch_bounds__(256)
    k_mv_post(const uint32_t* __restrict__ win_off, const uint32_t* __restrict__ mv_n,
              const uint32_t* __restrict__ mv_id, uint32_t n_genes, const uint32_t* __restrict__ post_ptr,
              uint32_t* __restrict__ mv_post, uint32_t* __restrict__ mv_plen) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_genes; g += warps) {
    const uint32_t off = win_off[g], n = mv_n[g];
    for (uint32_t e = lane; e < n; e += 32) {
      const uint32_t id = mv_id[off + e];
      const uint32_t lo = post_ptr[id];
      mv_post[off + e] = lo;
      mv_plen[off + e] = post_ptr[id + 1] - lo;
    }
  }
}

// ------------------------------------------------------------ query order
__global__ void k_order_count(const uint32_t* __restrict__ minhash, uint32_t n_genes, uint32_t shift,
                              uint32_t* __restrict__ count) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n_genes; g += gridDim.x * blockDim.x)
    atomicAdd(&count[minhash[g] >> shift], 1u);
}

__global__ void k_order_scatter(const uint32_t* __restrict__ minhash, uint32_t n_genes, uint32_t shift,
                                uint32_t* __restrict__ cursor, uint32_t* __restrict__ order) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n_genes; g += gridDim.x * blockDim.x)
    order[atomicAdd(&cursor[minhash[g] >> shift], 1u)] = g;
}

// ------------------------------------------------------------ small helpers
__global__ void k_gene_info(const int32_t* __restrict__ genome_ptr, uint32_t n_genomes,
                            const uint32_t* __restrict__ La, uint16_t* __restrict__ gene_genome,
                            uint32_t* __restrict__ ginfo) {
  for (uint32_t i = blockIdx.x; i < n_genomes; i += gridDim.x)
    for (int32_t g = genome_ptr[i] + (int32_t)threadIdx.x; g < genome_ptr[i + 1]; g += blockDim.x) {
      gene_genome[g] = (uint16_t)i;
      ginfo[g] = La[g] | (i << 16);
    }
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
    for (uint32_t e = lane; e < P.mv_n[g]; e += 32) {
      if (codes) codes[dst + e] = code_of_id[P.mv_id[off + e]];
      if (counts) counts[dst + e] = P.mv_cnt[off + e];
    }
  }
}

// Exact count of k-mer id in gene g (binary search in its multiplicity vector).
__device__ __forceinline__ uint32_t mv_count_of(const ProfilesView& P, uint32_t g, uint32_t id) {
  uint32_t lo = P.win_off[g], end = lo + P.mv_n[g], hi = end;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (P.mv_id[mid] < id) lo = mid + 1; else hi = mid;
  }
  return (lo < end && P.mv_id[lo] == id) ? P.mv_cnt[lo] : 0u;
}

__global__ void k_export_index(ProfilesView P, int32_t* __restrict__ genes, uint32_t* __restrict__ counts) {
  const uint32_t mask = (1u << P.cnt_bits) - 1u;
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

#define PD_LAUNCH(L, name, ...)             \
  do {                                      \
    cudaError_t e_ = launch_begin(L, name); \
    if (e_ != cudaSuccess) return e_;       \
    __VA_ARGS__;                            \
    e_ = launch_end(L, name);               \
    if (e_ != cudaSuccess) return e_;       \
  } while (0)

cudaError_t run_encode_mark(Launcher* L, const uint8_t* res, const int64_t* gene_ptr, uint32_t n_genes, int k,
                            unsigned long long* bitmap, DevErr* err, cudaStream_t s) {
  const unsigned grid = grid_for((uint64_t)n_genes * 32, kEncThreads, 152u * 16u);
  PD_LAUNCH(L, "encode_mark", k_encode_mark<<<grid, kEncThreads, 0, s>>>(res, gene_ptr, n_genes, k, bitmap, err));
  return cudaSuccess;
}

cudaError_t run_mv_build(Launcher* L, const uint8_t* res, const int64_t* gene_ptr, const uint32_t* win_off,
                         uint32_t n_genes, int k, const unsigned long long* bitmap, const uint32_t* word_rank,
                         uint32_t* mv_id, uint16_t* mv_cnt, uint32_t* mv_n, uint32_t* minhash,
                         const uint32_t* long_genes, uint32_t n_long, uint32_t* long_scratch,
                         const uint32_t* long_scratch_off, uint32_t max_smem_sort, cudaStream_t s) {
  const size_t smem = (size_t)max_smem_sort * sizeof(uint32_t);
  cudaError_t ea = cudaFuncSetAttribute(k_mv_build_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (ea != cudaSuccess) return ea;
  const unsigned grid = grid_for(n_genes, 1, 152u * 64u);
  PD_LAUNCH(L, "mv_build",
            k_mv_build_smem<<<grid, kMvThreads, smem, s>>>(res, gene_ptr, win_off, n_genes, k, bitmap, word_rank,
                                                            mv_id, mv_cnt, mv_n, minhash, max_smem_sort));
  if (n_long) {
    PD_LAUNCH(L, "mv_build_long",
              k_mv_build_long<<<grid_for(n_long, 1, 152u), kMvLongThreads, 0, s>>>(
                  res, gene_ptr, win_off, k, bitmap, word_rank, mv_id, mv_cnt, mv_n, minhash, long_genes, n_long,
                  long_scratch, long_scratch_off));
  }
  return cudaSuccess;
}

cudaError_t run_bucket_count(Launcher* L, const uint32_t* win_off, const uint32_t* mv_n, const uint32_t* mv_id,
                             uint32_t n_genes, uint32_t shift, uint32_t n_buckets, uint32_t* bucket_count,
                             cudaStream_t s) {
  const size_t smem = (size_t)n_buckets * sizeof(uint32_t);
  cudaError_t ea = cudaFuncSetAttribute(k_bucket_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (ea != cudaSuccess) return ea;
  PD_LAUNCH(L, "bucket_count",
            k_bucket_count<<<grid_for(n_genes, 64, 152u * 3u), kBucketThreads, smem, s>>>(
                win_off, mv_n, mv_id, n_genes, shift, n_buckets, bucket_count));
  return cudaSuccess;
}

cudaError_t run_bucket_scatter(Launcher* L, const uint32_t* win_off, const uint32_t* mv_n, const uint32_t* mv_id,
                               const uint16_t* mv_cnt, uint32_t n_genes, uint32_t shift, uint32_t n_buckets,
                               uint32_t* bucket_cursor, uint32_t cnt_bits, uint32_t cnt_cap,
                               unsigned long long* recs, cudaStream_t s) {
  const size_t smem = 2 * (size_t)n_buckets * sizeof(uint32_t);
  cudaError_t ea = cudaFuncSetAttribute(k_bucket_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (ea != cudaSuccess) return ea;
  PD_LAUNCH(L, "bucket_scatter",
            k_bucket_scatter<<<grid_for(n_genes, 64, 152u * 3u), kBucketThreads, smem, s>>>(
                win_off, mv_n, mv_id, mv_cnt, n_genes, shift, n_buckets, bucket_cursor, cnt_bits, cnt_cap, recs));
  return cudaSuccess;
}

cudaError_t run_bucket_fine(Launcher* L, const uint32_t* bucket_start, uint32_t n_buckets, uint32_t shift,
                            uint64_t n_ids, unsigned long long* recs, uint32_t* post_ptr, uint32_t* post,
                            uint32_t* max_posting, cudaStream_t s) {
  const size_t smem = 2 * ((size_t)1 << shift) * sizeof(uint32_t);
  cudaError_t ea = cudaFuncSetAttribute(k_bucket_fine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (ea != cudaSuccess) return ea;
  PD_LAUNCH(L, "bucket_fine",
            k_bucket_fine<<<grid_for(n_buckets, 1, 152u * 4u), kFineThreads, smem, s>>>(
                bucket_start, n_buckets, shift, n_ids, recs, post_ptr, post, max_posting));
  return cudaSuccess;
}

cudaError_t run_mv_post(Launcher* L, const uint32_t* win_off, const uint32_t* mv_n, const uint32_t* mv_id,
                        uint32_t n_genes, const uint32_t* post_ptr, uint32_t* mv_post, uint32_t* mv_plen,
                        cudaStream_t s) {
  PD_LAUNCH(L, "mv_post",
            k_mv_post<<<grid_for((uint64_t)n_genes * 32, 256, 152u * 16u), 256, 0, s>>>(
                win_off, mv_n, mv_id, n_genes, post_ptr, mv_post, mv_plen));
  return cudaSuccess;
}

cudaError_t run_order(Launcher* L, const uint32_t* minhash, uint32_t n_genes, uint32_t shift, uint32_t* count,
                      uint32_t* order, void* scan_tmp, cudaStream_t s) {
  const uint32_t n_b = 1u << (32 - shift);
  PD_LAUNCH(L, "order_count",
            k_order_count<<<grid_for(n_genes, 256, 152u * 8u), 256, 0, s>>>(minhash, n_genes, shift, count));
  cudaError_t e = scan_u32(L, count, n_b, count + n_b, scan_tmp, s);  // n_b + 1 prefix entries
  if (e != cudaSuccess) return e;
  PD_LAUNCH(L, "order_scatter",
            k_order_scatter<<<grid_for(n_genes, 256, 152u * 8u), 256, 0, s>>>(minhash, n_genes, shift,
                                                                             count + n_b, order));
  return cudaSuccess;
}

cudaError_t run_gene_info(Launcher* L, const int32_t* genome_ptr, uint32_t n_genomes, const uint32_t* La,
                          uint16_t* gene_genome, uint32_t* ginfo, cudaStream_t s) {
  PD_LAUNCH(L, "gene_info",
            k_gene_info<<<grid_for(n_genomes, 1, 152u * 8u), 256, 0, s>>>(genome_ptr, n_genomes, La, gene_genome,
                                                                         ginfo));
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
