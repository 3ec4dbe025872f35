// k_profiles.cu -- k-mer profiles on the device ("Multiplicity vector building
// phase", Algorithm 1, and the inverted index the sum-min kernel walks).
//
// Steps (one launch each):
//   encode_mark    letter -> 0..|G|-1 (|G| = 20 amino acids or 4
//                  nucleotides), base-|G| code of every window (Eq. (1):
//                  windows of exactly k letters), one bit per code in the
//                  dictionary's bit array over all |G|^k codes; letters
//                  outside the alphabet raise PD_ERR_ALPHABET.  Segmented
//                  datasets (independent problems profiled together) give each
//                  segment its own 20^k range of codes, code + segment * 20^k,
//                  so k-mers of different segments get different ids and never
//                  meet in a posting list.
//   (scan)         popcount prefix over the dictionary's 32-byte rank blocks
//                  (224 codes each): the dense id of a code is its rank among
//                  the codes present (an injective f that is ascending with
//                  the code, "Multiplicity vector building"), found with one
//                  sector read.
//   mv_build       per gene: ids of its windows counted in a shared-memory
//                  hash table, compacted into (id, multiplicity) pairs (Eqs.
//                  (2)-(3)), one index record per pair; also a min-hash.
//   (radix sort)   the inverted index is the transpose of the multiplicity
//                  vectors: the index records are sorted by k-mer id with a
//                  stable radix sort (k_radix.cu), which keeps each posting
//                  list in gene order.
//   mv_post        each multiplicity-vector entry gets its posting range, so
//                  the sum-min kernel reads list bounds from its own
//                  (coalesced) vector instead of the id offset table.
//   order          queries ordered by length bucket (at least 1024, 512, 256
//                  distinct k-mers, then the rest: longest first, so the
//                  persistent sum-min launch ends on short queries) and within
//                  a bucket by min-hash: genes that share their minimum hashed
//                  k-mer (likely homologs) run together and share posting
//                  lists in L2.
#include "pd_internal.cuh"

namespace pdg {
namespace {

constexpr int kEncThreads = 256;
constexpr int kMvThreads = 256;
constexpr int kMvLongThreads = 1024;
constexpr uint32_t kMvSmallCap = 2048;  // table slots of the shared-memory multiplicity-vector build
constexpr uint32_t kMvMidCap = 16384;   // ... of its 1024-thread variant (one block per SM)

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
                  uint32_t* __restrict__ dict, const uint16_t* __restrict__ gene_genome,
                  const unsigned long long* __restrict__ genome_code_base, const int64_t* __restrict__ gene_src,
                  int alpha, uint64_t n_res, DevErr* err) {
  __shared__ uint8_t lut[256];
  init_letter_table(lut, alpha);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_genes; g += warps) {
    const int64_t r0 = gene_src ? gene_src[g] : gene_ptr[g];
    const int64_t glen = gene_ptr[g + 1] - gene_ptr[g];
    // malformed offsets are reported by gene_windows; never read past them
    if (glen < 0 || r0 < 0 || (!gene_src && (uint64_t)(r0 + glen) > n_res)) continue;
    const uint32_t len = (uint32_t)glen;
    const uint8_t* s = res + r0;
    const unsigned long long base = genome_code_base ? genome_code_base[gene_genome[g]] : 0ull;
    for (uint32_t p = lane; p < len; p += 32) {
      if (lut[s[p]] >= (uint32_t)alpha) raise_error(err, PD_ERR_ALPHABET, (unsigned long long)(r0 + p));
    }
    // Each lane rolls the code over a contiguous run of windows: the code of
    // the window's last k-1 letters times alpha plus its last letter, then
    // minus the leading letter's share for the next window (Eq. (1)).  A
    // window is marked only if none of its letters is outside the alphabet.
    const uint32_t n_win = len >= (uint32_t)k ? len - (uint32_t)k + 1u : 0u;
    const uint32_t per = (n_win + 31u) / 32u;
    const uint32_t p0 = lane * per, p1 = min(n_win, p0 + per);
    if (p0 < p1) {
      const unsigned long long a = (unsigned long long)alpha;
      unsigned long long lead_w = 1;  // alpha^(k-1)
      for (int t = 1; t < k; ++t) lead_w *= a;
      unsigned long long code = 0;  // code of the k-1 letters before the next new letter
      int64_t last_bad = -1;        // position of the last letter outside the alphabet
      for (uint32_t q = p0; q + 1u < p0 + (uint32_t)k; ++q) {
        uint32_t c = lut[s[q]];
        if (c >= (uint32_t)alpha) {
          last_bad = q;
          c = 0;
        }
        code = code * a + c;
      }
      for (uint32_t p = p0; p < p1; ++p) {
        const uint32_t q = p + (uint32_t)k - 1u;
        uint32_t c = lut[s[q]];
        if (c >= (uint32_t)alpha) {
          last_bad = q;
          c = 0;
        }
        code = code * a + c;
        if (last_bad < (int64_t)p) {
          unsigned long long blk;
          uint32_t w, bit;
          dict_locate(code + base, &blk, &w, &bit);
          atomicOr(&dict[blk * 8 + w], 1u << bit);
        }
        uint32_t lead = lut[s[p]];
        code -= (unsigned long long)(lead < (uint32_t)alpha ? lead : 0u) * lead_w;
      }
    }
  }
}

// ------------------------------------------------------------ gene windows
__host__ __device__ __forceinline__ uint32_t mv_table_cap(uint32_t La);

__global__ void k_gene_windows(const int64_t* __restrict__ gene_ptr, uint32_t n_genes, uint64_t n_res, int check_end,
                               int k, uint32_t* __restrict__ La, uint32_t* __restrict__ mid_list,
                               uint32_t* __restrict__ long_list, unsigned long long* __restrict__ long_off,
                               uint32_t* counts, unsigned long long* long_total, DevErr* err) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n_genes; g += gridDim.x * blockDim.x) {
    const int64_t r0 = gene_ptr[g], r1 = gene_ptr[g + 1];
    const bool bad = r1 < r0 || (g == 0 && r0 != 0) || (check_end && g + 1 == n_genes && (uint64_t)r1 != n_res);
    if (bad) {
      raise_error(err, PD_ERR_ARG, g);
      La[g] = 0;
      continue;
    }
    const int64_t len = r1 - r0;
    uint64_t w = len >= k ? (uint64_t)(len - k + 1) : 0;
    if (w > PD_MAX_WINDOWS) {
      raise_error(err, PD_ERR_GENE_TOO_LONG, g);
      w = 0;
    }
    La[g] = (uint32_t)w;
    const uint32_t cap = mv_table_cap((uint32_t)w);
    if (cap > kMvMidCap) {
      const uint32_t x = atomicAdd(&counts[1], 1u);
      long_list[x] = g;
      long_off[x] = atomicAdd(long_total, (unsigned long long)cap);
    } else if (cap > kMvSmallCap) {
      mid_list[atomicAdd(&counts[0], 1u)] = g;
    }
  }
}

__global__ void k_narrow_u64(const unsigned long long* __restrict__ in, uint64_t n, uint32_t* __restrict__ out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)in[i];
}

// ------------------------------------------------------------ mv_build
// Multiplicity vector of gene g (Eqs. (2)-(3)): the dense ids of its windows
// are counted in an open-addressing table of 64-bit slots (id << 32 | count)
// of `cap` slots (a power of two, at least 1.5 x La), then the occupied slots
// are compacted into the gene's window range.  The entries of one vector are
// in table order: nothing downstream depends on their order (sums commute,
// posting lists are sorted by gene later, and the export hook sorts by code).
// Besides (id, count) the gene emits one 64-bit record per entry for the
// index build, (id << 32) | packed posting, and marks the unused tail of its
// window range with all-ones records.  Called by every thread of the block.
__device__ __forceinline__ void mv_build_one(uint32_t g, unsigned long long* table, uint32_t cap,
                                             const uint8_t* __restrict__ lut, uint32_t* warp_tmp,
                                             const uint8_t* __restrict__ res, const int64_t* __restrict__ gene_ptr,
                                             const uint32_t* __restrict__ win_off, int k,
                                             const uint32_t* __restrict__ dict, const MvOut& M) {
  constexpr unsigned long long kFree = ~0ull;
  const uint32_t off = win_off[g];
  const uint32_t La = win_off[g + 1] - off;
  const uint8_t* s = res + (M.gene_src ? M.gene_src[g] : gene_ptr[g]);
  const unsigned long long base = M.genome_code_base ? M.genome_code_base[M.gene_genome[g]] : 0ull;
  for (uint32_t h = threadIdx.x; h < cap; h += blockDim.x) table[h] = kFree;
  __syncthreads();
  for (uint32_t p = threadIdx.x; p < La; p += blockDim.x) {
    unsigned long long code = 0;
    for (int t = 0; t < k; ++t) {
      const uint32_t c = lut[s[p + t]];
      code = code * (unsigned long long)M.alpha + (c < (uint32_t)M.alpha ? c : 0u);
    }
    if (M.frozen && !dict_has(dict, code + base)) continue;  // not in that dictionary
    const uint32_t id = dict_rank(dict, code + base);
    uint32_t h = mix32(id) & (cap - 1u);
    uint32_t probe = 0;
    for (; probe < cap; ++probe) {  // a free slot always exists: cap > La >= distinct ids
      const unsigned long long cur = *((volatile unsigned long long*)&table[h]);
      if (cur != kFree && (uint32_t)(cur >> 32) == id) {
        atomicAdd(&table[h], 1ull);
        break;
      }
      if (cur == kFree) {
        const unsigned long long prev = atomicCAS(&table[h], kFree, ((unsigned long long)id << 32) | 1ull);
        if (prev == kFree) break;
        if ((uint32_t)(prev >> 32) == id) {
          atomicAdd(&table[h], 1ull);
          break;
        }
      }
      h = (h + 1u) & (cap - 1u);
    }
    if (probe == cap) raise_error(M.err, PD_ERR_INTERNAL, g);  // unreachable by the bound above
  }
  __syncthreads();
  // compaction of the occupied slots (interleaved: slot = i * blockDim + tid)
  uint32_t mine = 0;
  for (uint32_t h = threadIdx.x; h < cap; h += blockDim.x) mine += table[h] != kFree ? 1u : 0u;
  uint32_t E;
  uint32_t pos = block_exclusive_scan(mine, warp_tmp, &E);
  uint32_t mh = kEmpty;
  for (uint32_t h = threadIdx.x; h < cap; h += blockDim.x) {
    const unsigned long long v = table[h];
    if (v == kFree) continue;
    const uint32_t id = (uint32_t)(v >> 32), c = (uint32_t)v;
    M.mv_id[off + pos] = id;
    M.mv_cnt[off + pos] = (uint16_t)c;
    if (M.rec) M.rec[off + pos] = ((unsigned long long)id << 32) | (g << M.cnt_bits) | (c < M.cnt_cap ? c : M.cnt_cap);
    mh = min(mh, mix32(id));
    ++pos;
  }
  if (M.rec)
    for (uint32_t p = E + threadIdx.x; p < La; p += blockDim.x) M.rec[off + p] = kFree;
  // block minimum of the hashed ids (warp_tmp is free again after the scan)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mh = min(mh, __shfl_xor_sync(0xffffffffu, mh, o));
  if (threadIdx.x == 0) warp_tmp[0] = kEmpty;
  __syncthreads();
  if ((threadIdx.x & 31u) == 0) atomicMin(&warp_tmp[0], mh);
  __syncthreads();
  if (threadIdx.x == 0) {
    M.mv_n[g] = E;
    // query order key: optionally a length bucket (longest first) in the top
    // two bits, then the min-hash
    const uint32_t lb = E >= 1024u ? 0u : (E >= 512u ? 1u : (E >= 256u ? 2u : 3u));
    if (M.minhash) M.minhash[g] = M.length_buckets ? (lb << 30) | (warp_tmp[0] >> 2) : warp_tmp[0];
  }
  __syncthreads();
}

__host__ __device__ __forceinline__ uint32_t mv_table_cap(uint32_t La) {
  const uint32_t c = next_pow2(La + La / 2 + 1);
  return c < 64 ? 64 : c;
}

// Genes whose table fits `max_cap` slots of shared memory: all genes with a
// table of at most max_cap slots (list == nullptr), or the listed genes.
template <int kThreads>
__global__ void __launch_bounds__(kThreads)
    k_mv_build_smem(const uint8_t* __restrict__ res, const int64_t* __restrict__ gene_ptr,
                    const uint32_t* __restrict__ win_off, uint32_t n_genes, int k,
                    const uint32_t* __restrict__ dict, MvOut M,
                    uint32_t max_cap, const uint32_t* __restrict__ list, uint32_t n_list) {
  extern __shared__ unsigned long long table[];
  __shared__ uint8_t lut[256];
  __shared__ uint32_t warp_tmp[kThreads / 32 + 1];
  init_letter_table(lut, M.alpha);
  const uint32_t n = list ? n_list : n_genes;
  for (uint32_t x = blockIdx.x; x < n; x += gridDim.x) {
    const uint32_t g = list ? list[x] : x;
    const uint32_t cap = mv_table_cap(win_off[g + 1] - win_off[g]);
    if (cap > max_cap) continue;  // uniform over the block: built by a later launch
    mv_build_one(g, table, cap, lut, warp_tmp, res, gene_ptr, win_off, k, dict, M);
  }
}

// Genes too long for shared memory: tables in global scratch (one per gene).
__global__ void __launch_bounds__(kMvLongThreads)
    k_mv_build_long(const uint8_t* __restrict__ res, const int64_t* __restrict__ gene_ptr,
                    const uint32_t* __restrict__ win_off, int k, const uint32_t* __restrict__ dict, MvOut M,
                    const uint32_t* __restrict__ long_genes,
                    uint32_t n_long, unsigned long long* scratch, const unsigned long long* __restrict__ scratch_off) {
  __shared__ uint8_t lut[256];
  __shared__ uint32_t warp_tmp[kMvLongThreads / 32 + 1];
  init_letter_table(lut, M.alpha);
  for (uint32_t x = blockIdx.x; x < n_long; x += gridDim.x) {
    const uint32_t g = long_genes[x];
    mv_build_one(g, scratch + scratch_off[x], mv_table_cap(win_off[g + 1] - win_off[g]), lut, warp_tmp, res,
                 gene_ptr, win_off, k, dict, M);
  }
}

// Every multiplicity-vector entry gets its posting range [mv_post, +mv_plen);
// the longest list length goes to *max_posting and, if join is not null, the
// sum of the entries' list lengths -- the postings an all-against-all walk
// visits -- is added to *join.
__global__ void __launch_bounds__(256)
    k_mv_post(const uint32_t* __restrict__ win_off, const uint32_t* __restrict__ mv_n,
              const uint32_t* __restrict__ mv_id, uint32_t n_genes, const uint32_t* __restrict__ post_ptr,
              uint32_t* __restrict__ mv_post, uint32_t* __restrict__ mv_plen, uint32_t* __restrict__ max_posting,
              unsigned long long* __restrict__ join) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  uint32_t m = 0;
  unsigned long long jsum = 0;
  for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_genes; g += warps) {
    const uint32_t off = win_off[g], n = mv_n[g];
    // four entries per lane in flight: their ids, then their list bounds
    for (uint32_t e0 = lane; e0 < n; e0 += 128) {
      uint32_t id[4], lo[4], hi[4];
#pragma unroll
      for (uint32_t j = 0; j < 4; ++j) id[j] = e0 + 32 * j < n ? mv_id[off + e0 + 32 * j] : 0u;
#pragma unroll
      for (uint32_t j = 0; j < 4; ++j) {
        lo[j] = hi[j] = 0;
        if (e0 + 32 * j < n) {
          lo[j] = post_ptr[id[j]];
          hi[j] = post_ptr[id[j] + 1];
        }
      }
#pragma unroll
      for (uint32_t j = 0; j < 4; ++j) {
        if (e0 + 32 * j < n) {
          mv_post[off + e0 + 32 * j] = lo[j];
          mv_plen[off + e0 + 32 * j] = hi[j] - lo[j];
          m = max(m, hi[j] - lo[j]);
          jsum += hi[j] - lo[j];
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    jsum += __shfl_xor_sync(0xffffffffu, jsum, o);
  }
  if (lane == 0 && m) atomicMax(max_posting, m);
  if (lane == 0 && join && jsum) atomicAdd(join, jsum);
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

// Code of every dense id: the set bits of each dictionary block, in order.
__global__ void k_select_codes(const uint32_t* __restrict__ dict, uint64_t n_blocks,
                               unsigned long long* __restrict__ code_of_id) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_blocks;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t id = dict[i * 8];
    for (uint32_t w = 1; w < 8; ++w) {
      uint32_t bits = dict[i * 8 + w];
      while (bits) {
        const int bit = __ffs((int)bits) - 1;
        code_of_id[id++] = i * kDictBits + (w - 1u) * 32u + (unsigned long long)bit;
        bits &= bits - 1u;
      }
    }
  }
}

// Export of the multiplicity vectors in ascending code order (inspection
// hook): each gene's (code << 16 | count) keys go to a power-of-two padded
// scratch region, one block sorts each region, then the keys are unpacked.
__global__ void k_export_mv_keys(ProfilesView P, const unsigned long long* __restrict__ pad_off,
                                 const unsigned long long* __restrict__ code_of_id, unsigned long long* __restrict__ pad) {
  for (uint32_t g = blockIdx.x; g < P.n_genes; g += gridDim.x) {
    const uint32_t off = P.win_off[g], n = P.mv_n[g];
    const unsigned long long o = pad_off[g], n2 = pad_off[g + 1] - o;
    for (uint32_t e = threadIdx.x; e < n2; e += blockDim.x)
      pad[o + e] = e < n ? (code_of_id[P.mv_id[off + e]] << 16) | P.mv_cnt[off + e] : ~0ull;
  }
}

__global__ void __launch_bounds__(512) k_export_mv_sort(uint32_t n_genes, const unsigned long long* __restrict__ pad_off,
                                                        unsigned long long* pad) {
  for (uint32_t g = blockIdx.x; g < n_genes; g += gridDim.x) {
    const unsigned long long o = pad_off[g];
    const uint32_t n2 = (uint32_t)(pad_off[g + 1] - o);
    if (n2 > 1) block_bitonic_sort(pad + o, n2);
    __syncthreads();
  }
}

__global__ void k_export_mv(ProfilesView P, const unsigned long long* __restrict__ mv_ptr,
                            const unsigned long long* __restrict__ pad_off, const unsigned long long* __restrict__ pad,
                            unsigned long long* __restrict__ codes, uint32_t* __restrict__ counts) {
  for (uint32_t g = blockIdx.x; g < P.n_genes; g += gridDim.x) {
    const unsigned long long o = pad_off[g], dst = mv_ptr[g];
    for (uint32_t e = threadIdx.x; e < P.mv_n[g]; e += blockDim.x) {
      const unsigned long long v = pad[o + e];
      if (codes) codes[dst + e] = v >> 16;
      if (counts) counts[dst + e] = (uint32_t)(v & 0xFFFFu);
    }
  }
}

// Exact count of k-mer id in gene g (its multiplicity vector is unordered).
__device__ __forceinline__ uint32_t mv_count_of(const ProfilesView& P, uint32_t g, uint32_t id) {
  const uint32_t off = P.win_off[g], n = P.mv_n[g];
  for (uint32_t e = 0; e < n; ++e)
    if (P.mv_id[off + e] == id) return P.mv_cnt[off + e];
  return 0u;
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
                            uint32_t* dict, const uint16_t* gene_genome,
                            const unsigned long long* genome_code_base, const int64_t* gene_src, int alpha,
                            uint64_t n_res, DevErr* err, cudaStream_t s) {
  const unsigned grid = grid_for((uint64_t)n_genes * 32, kEncThreads, 152u * 16u);
  PD_LAUNCH(L, "encode_mark", k_encode_mark<<<grid, kEncThreads, 0, s>>>(res, gene_ptr, n_genes, k, dict,
                                                                        gene_genome, genome_code_base, gene_src,
                                                                        alpha, n_res, err));
  return cudaSuccess;
}

cudaError_t run_gene_windows(Launcher* L, const int64_t* gene_ptr, uint32_t n_genes, uint64_t n_res, int check_end,
                             int k, uint32_t* La, uint32_t* mid_list, uint32_t* long_list,
                             unsigned long long* long_off, uint32_t* counts, unsigned long long* long_total,
                             DevErr* err, cudaStream_t s) {
  PD_LAUNCH(L, "gene_windows",
            k_gene_windows<<<grid_for(n_genes, 256, 152u * 8u), 256, 0, s>>>(gene_ptr, n_genes, n_res, check_end, k,
                                                                            La, mid_list, long_list, long_off,
                                                                            counts, long_total, err));
  return cudaSuccess;
}

cudaError_t run_narrow_u64(Launcher* L, const unsigned long long* in, uint64_t n, uint32_t* out, cudaStream_t s) {
  PD_LAUNCH(L, "narrow_u64", k_narrow_u64<<<grid_for(n, 256, 152u * 8u), 256, 0, s>>>(in, n, out));
  return cudaSuccess;
}

cudaError_t run_mv_build(Launcher* L, const uint8_t* res, const int64_t* gene_ptr, const uint32_t* win_off,
                         uint32_t n_genes, int k, const uint32_t* dict, const MvOut& M, const uint32_t* mid_genes, uint32_t n_mid, const uint32_t* long_genes,
                         uint32_t n_long, unsigned long long* long_scratch, const unsigned long long* long_scratch_off,
                         cudaStream_t s) {
  const size_t smem1 = (size_t)kMvSmallCap * 8, smem2 = (size_t)kMvMidCap * 8;
  cudaError_t ea = cudaFuncSetAttribute(k_mv_build_smem<kMvThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem1);
  if (ea != cudaSuccess) return ea;
  ea = cudaFuncSetAttribute(k_mv_build_smem<kMvLongThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
  if (ea != cudaSuccess) return ea;
  PD_LAUNCH(L, "mv_build",
            k_mv_build_smem<kMvThreads><<<grid_for(n_genes, 1, 152u * 64u), kMvThreads, smem1, s>>>(
                res, gene_ptr, win_off, n_genes, k, dict, M, kMvSmallCap, nullptr, 0u));
  if (n_mid) {
    PD_LAUNCH(L, "mv_build_mid",
              k_mv_build_smem<kMvLongThreads><<<grid_for(n_mid, 1, 152u), kMvLongThreads, smem2, s>>>(
                  res, gene_ptr, win_off, n_genes, k, dict, M, kMvMidCap, mid_genes, n_mid));
  }
  if (n_long) {
    PD_LAUNCH(L, "mv_build_long",
              k_mv_build_long<<<grid_for(n_long, 1, 152u), kMvLongThreads, 0, s>>>(
                  res, gene_ptr, win_off, k, dict, M, long_genes, n_long, long_scratch,
                  long_scratch_off));
  }
  return cudaSuccess;
}

uint32_t mv_build_table_cap(uint32_t La) { return mv_table_cap(La); }

cudaError_t run_mv_post(Launcher* L, const uint32_t* win_off, const uint32_t* mv_n, const uint32_t* mv_id,
                        uint32_t n_genes, const uint32_t* post_ptr, uint32_t* mv_post, uint32_t* mv_plen,
                        uint32_t* max_posting, unsigned long long* join, cudaStream_t s) {
  PD_LAUNCH(L, "mv_post",
            k_mv_post<<<grid_for((uint64_t)n_genes * 32, 256, 152u * 16u), 256, 0, s>>>(
                win_off, mv_n, mv_id, n_genes, post_ptr, mv_post, mv_plen, max_posting, join));
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

cudaError_t run_select_codes(Launcher* L, const uint32_t* dict, uint64_t n_blocks, unsigned long long* code_of_id,
                             cudaStream_t s) {
  PD_LAUNCH(L, "select_codes",
            k_select_codes<<<grid_for(n_blocks, 256, 152u * 16u), 256, 0, s>>>(dict, n_blocks, code_of_id));
  return cudaSuccess;
}

cudaError_t run_export_mv(Launcher* L, const ProfilesView& P, const unsigned long long* mv_ptr,
                          const unsigned long long* pad_off, unsigned long long* pad,
                          const unsigned long long* code_of_id, unsigned long long* codes, uint32_t* counts,
                          cudaStream_t s) {
  const unsigned grid = grid_for(P.n_genes, 1, 152u * 16u);
  PD_LAUNCH(L, "export_mv_keys", k_export_mv_keys<<<grid, 256, 0, s>>>(P, pad_off, code_of_id, pad));
  PD_LAUNCH(L, "export_mv_sort", k_export_mv_sort<<<grid, 512, 0, s>>>(P.n_genes, pad_off, pad));
  PD_LAUNCH(L, "export_mv", k_export_mv<<<grid, 256, 0, s>>>(P, mv_ptr, pad_off, pad, codes, counts));
  return cudaSuccess;
}

cudaError_t run_export_index(Launcher* L, const ProfilesView& P, int32_t* genes, uint32_t* counts, cudaStream_t s) {
  PD_LAUNCH(L, "export_index",
            k_export_index<<<grid_for(P.n_entries, 256, 152u * 16u), 256, 0, s>>>(P, genes, counts));
  return cudaSuccess;
}

}  // namespace pdg
