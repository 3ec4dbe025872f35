// pd_internal.cuh -- shared declarations of the CUDA implementation of pd.h.
//
// Device data layout of a profiled dataset (all arrays in HBM, built once by
// pd_build_profiles and read by every later call):
//
//   gene g (global id, 0..G-1) has La[g] = max(0, |g|-k+1) k-mer windows.
//   win_off[G+1]   uint32  exclusive prefix of La: window range of each gene.
//   mv_n[G]        uint32  distinct k-mers of the gene (E_g <= La[g]).
//   mv_id[W]       uint32  dense k-mer id, gene g at win_off[g] .. +mv_n[g]
//                          (the multiplicity vector of Algorithm 1, stored in
//                          the gene's window range: "padded CSR"; the entries
//                          of one gene are unordered).
//   mv_cnt[W]      uint16  multiplicity of that k-mer in the gene.
//   mv_post[W],    uint32  posting range of that k-mer (copied from post_ptr so
//   mv_plen[W]             a query reads its list bounds with its own vector).
//   gene_genome[G] uint16  genome of each gene; ginfo[G] = La | genome << 16.
//   dict[8 * ceil(20^k / 224)] uint32  the dictionary, one bit per possible
//                          k-mer code in rank blocks of 32 bytes (one DRAM
//                          sector): block b covers codes 224b .. 224b+223,
//                          word 0 = number of codes present in blocks 0..b-1,
//                          words 1..7 = the block's bits (code 224b + j is bit
//                          j % 32 of word 1 + j / 32).  The dense id of a
//                          present code is word 0 plus the set bits before it
//                          in its block (ascending in code order), read with
//                          one sector per lookup.
//   post_ptr[D+1]  uint32  inverted index: postings of id w are
//   post[E]        uint32  post[post_ptr[w] .. post_ptr[w+1]), ascending by
//                          gene, each packed as (gene << cnt_bits) | min(count,
//                          cnt_cap) with cnt_bits = 32 - bits(G-1).  A count
//                          equal to cnt_cap is saturated; the exact value is
//                          in the gene's multiplicity vector.
//   order[G]       uint32  all-pairs query order: genes grouped by the top bits
//                          of their min-hash (minimum of a hash of their k-mer
//                          ids), so likely homologs run together.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pd.h"

namespace pdg {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;

// ---------------------------------------------------------------- dictionary
constexpr uint32_t kDictBits = 224;  // codes per 32-byte rank block
__host__ __device__ __forceinline__ uint64_t dict_blocks(uint64_t n_codes) {
  return (n_codes + kDictBits - 1) / kDictBits;
}
// Block of a code, and the code's word (1..7) and bit inside it.
__device__ __forceinline__ void dict_locate(unsigned long long code, unsigned long long* blk, uint32_t* word,
                                            uint32_t* bit) {
  const unsigned long long b = code / kDictBits;
  const uint32_t off = (uint32_t)(code - b * kDictBits);
  *blk = b;
  *word = 1u + (off >> 5);
  *bit = off & 31u;
}
__device__ __forceinline__ bool dict_has(const uint32_t* __restrict__ dict, unsigned long long code) {
  unsigned long long b;
  uint32_t w, bit;
  dict_locate(code, &b, &w, &bit);
  return (dict[b * 8 + w] >> bit) & 1u;
}
// Dense id of a present code: the block's base plus the set bits before it.
__device__ __forceinline__ uint32_t dict_rank(const uint32_t* __restrict__ dict, unsigned long long code) {
  unsigned long long b;
  uint32_t w, bit;
  dict_locate(code, &b, &w, &bit);
  const uint4* q = reinterpret_cast<const uint4*>(dict + b * 8);
  const uint4 lo = q[0], hi = q[1];
  const uint32_t words[7] = {lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
  uint32_t r = lo.x;
#pragma unroll
  for (uint32_t j = 0; j < 7; ++j) {
    const uint32_t m = j + 1u < w ? 0xFFFFFFFFu : (j + 1u == w ? (1u << bit) - 1u : 0u);
    r += (uint32_t)__popc(words[j] & m);
  }
  return r;
}
constexpr int kAlphabetSize = 20;

// ---------------------------------------------------------------- errors
// Device error block: kernels record the first error code and a detail value
// (e.g. the offending residue position) and skip the faulty item.
struct DevErr {
  int code;
  int pad;
  unsigned long long detail;
};

__device__ __forceinline__ void raise_error(DevErr* e, int code, unsigned long long detail) {
  if (atomicCAS(&e->code, 0, code) == 0) e->detail = detail;
}

// ---------------------------------------------------------------- helpers
__host__ __device__ __forceinline__ uint32_t next_pow2(uint32_t x) {
  if (x <= 1) return 1;
  --x;
  x |= x >> 1;
  x |= x >> 2;
  x |= x >> 4;
  x |= x >> 8;
  x |= x >> 16;
  return x + 1;
}

// Letter -> 0..alpha-1, 255 otherwise; built per block.  alpha 20: amino
// acids in ACDEFGHIKLMNPQRSTVWY order; alpha 4: nucleotides in ACGT order.
__device__ __forceinline__ void init_letter_table(uint8_t* lut, int alpha) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) lut[i] = 255;
  __syncthreads();
  const char* letters = alpha == 4 ? "ACGT" : "ACDEFGHIKLMNPQRSTVWY";
  if ((int)threadIdx.x < alpha) lut[(uint8_t)letters[threadIdx.x]] = (uint8_t)threadIdx.x;
  __syncthreads();
}

// Ascending bitonic sort of n (a power of two) keys by the whole block.
template <typename K>
__device__ __forceinline__ void block_bitonic_sort(K* a, uint32_t n) {
  for (uint32_t size = 2; size <= n; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < (n >> 1); i += blockDim.x) {
        uint32_t lo = 2 * i - (i & (stride - 1));
        uint32_t hi = lo + stride;
        bool asc = (lo & size) == 0;
        K x = a[lo], y = a[hi];
        if ((x > y) == asc) {
          a[lo] = y;
          a[hi] = x;
        }
      }
      __syncthreads();
    }
  }
}

// Inclusive warp scan of v.
__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t v) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= (uint32_t)o) v += y;
  }
  return v;
}

// Exclusive block scan; `warp_tmp` holds at least blockDim.x/32 + 1 words.
// Returns the exclusive prefix of v; *total receives the block sum.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tmp, uint32_t* total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t n_warps = (blockDim.x + 31) >> 5;
  uint32_t inc = warp_inclusive_scan(v);
  if (lane == 31) warp_tmp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = (lane < n_warps) ? warp_tmp[lane] : 0u;
    uint32_t wi = warp_inclusive_scan(w);
    if (lane < n_warps) warp_tmp[lane] = wi - w;
    if (lane == n_warps - 1) warp_tmp[n_warps] = wi;
  }
  __syncthreads();
  uint32_t r = warp_tmp[warp] + inc - v;
  *total = warp_tmp[n_warps];
  __syncthreads();
  return r;
}

// Exact ratio order: s1/d1 > s2/d2 by 64-bit cross-multiplication.
__host__ __device__ __forceinline__ bool ratio_greater(uint32_t s1, uint32_t d1, uint32_t s2, uint32_t d2) {
  return (uint64_t)s1 * (uint64_t)d2 > (uint64_t)s2 * (uint64_t)d1;
}
__host__ __device__ __forceinline__ bool ratio_equal(uint32_t s1, uint32_t d1, uint32_t s2, uint32_t d2) {
  return (uint64_t)s1 * (uint64_t)d2 == (uint64_t)s2 * (uint64_t)d1;
}

// ---------------------------------------------------------------- views
struct ProfilesView {
  int k;
  uint32_t n_genes, n_genomes;
  uint64_t n_windows, n_distinct, n_entries;
  uint32_t cnt_bits, cnt_cap, max_posting;
  uint64_t n_join;              // postings the all-against-all walk visits (sum over entries of list length)
  const uint32_t* win_off;      // [G+1] window range of each gene
  const uint32_t* mv_n;         // [G]   distinct k-mers of each gene
  const uint32_t* mv_id;        // [W]   multiplicity vectors: dense ids
  const uint16_t* mv_cnt;       // [W]   multiplicities
  const uint32_t* mv_post;      // [W]   posting-list start of each entry's id
  const uint32_t* mv_plen;      // [W]   posting-list length of each entry's id
  const uint32_t* La;           // [G]   windows per gene
  const uint16_t* gene_genome;  // [G]   genome of each gene
  const uint32_t* ginfo;        // [G]   La | genome << 16
  const int32_t* genome_ptr;    // [n+1] device copy
  const uint32_t* dict;         // [8 * n_dict_blocks] dictionary rank blocks
  uint64_t n_dict_blocks;
  const uint32_t* post_ptr;     // [D+1]
  const uint32_t* post;         // [E]   packed postings
  const uint32_t* order;        // [G]   all-pairs query order (min-hash buckets)
  // External queries (null = queries are genes of this dataset): genes
  // profiled against this dataset's dictionary but not part of it; query a
  // reads its vector from these arrays (indexed like the ones above, by the
  // query's own numbering) while targets stay this dataset's genes.
  const uint32_t* q_win_off;
  const uint32_t* q_mv_n;
  const uint32_t* q_mv_id;
  const uint16_t* q_mv_cnt;
  const uint32_t* q_mv_post;
  const uint32_t* q_mv_plen;
  const uint32_t* q_La;
};

// Target selection of one sum-min launch.
//   all_pairs = 1: query index x is gene order[x] (or q0 + x without an order)
//                  and each query targets every genome except its own; its
//                  output row is its gene id.
//   all_pairs = 0: query index x < nA is gene qa0 + x targeting genes
//                  [ta0, ta1); index x >= nA is gene qb0 + (x - nA) targeting
//                  [tb0, tb1); the output row is x.
struct QuerySet {
  int all_pairs;
  const uint32_t* order;
  uint32_t q0, n_queries;
  // Sharded all-pairs form (n_shards = 0: off): only the query genes g with
  // g mod n_shards == shard are computed (the others are skipped before any
  // work), so the shards partition the genes whatever the query order.
  uint32_t n_shards, shard;
  // Symmetric all-pairs form (symbest not null): each unordered genome pair is
  // walked from one side.  Query a walks only the targets in genomes after its
  // own; for every candidate b it keeps the best (s, den, a) of b over a's
  // genome at symbest[genome(a) * n_genes + b] -- the reverse-direction
  // maximum, packed s << 48 | den << 31 | a -- and lists exact ties of that
  // maximum as the pair of words (b << 32 | a, s) in tie_rec (tie_cap pairs;
  // the count keeps counting past it).
  unsigned long long* symbest;
  unsigned long long* tie_rec;
  unsigned long long* tie_count;
  unsigned long long tie_cap;
  uint32_t qa0, nA, ta0, ta1;
  uint32_t qb0, tb0, tb1;
  // Served queries (all-pairs form; null = off).  tgt_end[genome of the
  // query]: only genes below it are targets.  colbest: for every target gene
  // b and query genome g, the best (s << 32 | den) of b over the genes of g,
  // at colbest[b * col_stride + (g - col_genome0)] (the reverse-direction
  // Best Hit maximum, kept by compare-and-swap).
  const uint32_t* tgt_end;
  unsigned long long* colbest;
  uint32_t col_genome0, col_stride;
  // Within-genome form (pair indexing, row = q0 + query): each query gene is
  // compared with the other genes of its own genome (not with itself).
  int paralog;
  // Listed form (pair indexing, row = query): query x is gene q_gene[x] and
  // targets genes [q_t0[x], q_t1[x]) -- many genome pairs in one launch.
  const uint32_t* q_gene;
  const uint32_t* q_t0;
  const uint32_t* q_t1;
  // External queries (with the q_* arrays of the view): the genome of each
  // query gene among the queries' own genomes; it has no own-genome targets,
  // tgt_end and the colbest column are indexed by it.
  const uint32_t* q_genome;
  // Candidate filters (filter != 0): the length threshold theta = theta_num /
  // theta_den of Eq. (6) and the directional threshold tau = tau_num /
  // tau_den of Eq. (7); a numerator of 0 turns a filter off.
  int filter;
  uint32_t theta_num, theta_den, tau_num, tau_den;
  // Posting walk of tier 1 (PD_WALK_*): automatic (from the join per vector
  // entry), merge-path, or warp-cooperative.
  uint32_t walk;
};

struct HitsOut {
  uint32_t* out_b;                   // global target gene id
  uint32_t* out_s;                   // sum-min
  unsigned long long out_cap;        // capacity of out_b / out_s
  unsigned long long* cursor;        // append cursor (keeps counting past cap)
  unsigned long long* row_off;       // per output row
  uint32_t* row_len;                 // per output row
  uint32_t* def1;                    // queries deferred by tier 1 ...
  uint32_t* n_def1;
  uint32_t* def2;                    // ... and by tier 2
  uint32_t* n_def2;
  unsigned long long* walked;        // postings visited
};

// Global-memory scratch of the last tier (per block: table, occupied-slot
// list and hits).
struct BigScratch {
  uint32_t* keys;        // n_ctas * cap
  uint32_t* vals;        // n_ctas * cap
  uint32_t* used;        // n_ctas * cap
  unsigned long long* out;  // n_ctas * out_cap
  uint32_t cap;          // power of two
  uint32_t out_cap;
  uint32_t* vpa = nullptr;  // filtered queries: n_ctas * cap directional sums (query side)
  uint32_t* vpb = nullptr;  // ... (target side)
};

// Queries of one sum-min launch: the range 0..n_queries-1 (first tier) or a
// list of query indices with its count in device memory (later tiers).
struct TierIO {
  const uint32_t* in_list;
  const uint32_t* in_count;
  uint32_t* def_list;   // deferred queries (nullptr in the last tier)
  uint32_t* def_count;
};

// ---------------------------------------------------------------- launchers
// Every launcher enqueues on `stream` and returns the launch error (if any).
struct Launcher;  // opaque: pd_ctx side (timing + launch counting)
cudaError_t launch_begin(Launcher* L, const char* name);
cudaError_t launch_end(Launcher* L, const char* name);

// scans (k_scan.cu)
size_t scan_temp_bytes(uint64_t n);
// Rank bases of the dictionary: word 0 of each of the n_blocks blocks gets
// the set bits of the blocks before it; *total gets the number of codes.
cudaError_t scan_dict_blocks(Launcher* L, uint32_t* dict, uint64_t n_blocks, uint32_t* total, void* temp,
                             cudaStream_t s);
cudaError_t scan_u32(Launcher* L, const uint32_t* in, uint64_t n, uint32_t* out_excl_np1, void* temp,
                     cudaStream_t s);
cudaError_t scan_u32_to_u64(Launcher* L, const uint32_t* in, uint64_t n, unsigned long long* out_excl_np1,
                            void* temp, cudaStream_t s);

// profiles (k_profiles.cu)
// Gene offsets -> window counts on the device.  Checks every gene (offsets
// from 0, non-decreasing, ending at n_res unless check_end is 0; at most
// PD_MAX_WINDOWS windows), recording PD_ERR_ARG / PD_ERR_GENE_TOO_LONG with
// the gene as detail (such a gene gets La 0); lists the genes whose vector
// table exceeds the small (mid) and the large (long) shared-memory build, with
// a scratch offset for each long gene.  counts: [n_mid, n_long] (uint32) and
// long_total (uint64, after them, 8-byte aligned).
cudaError_t run_gene_windows(Launcher* L, const int64_t* gene_ptr, uint32_t n_genes, uint64_t n_res, int check_end,
                             int k, uint32_t* La, uint32_t* mid_list, uint32_t* long_list,
                             unsigned long long* long_off, uint32_t* counts, unsigned long long* long_total,
                             DevErr* err, cudaStream_t s);
// u64 -> u32 copy of n values.
cudaError_t run_narrow_u64(Launcher* L, const unsigned long long* in, uint64_t n, uint32_t* out, cudaStream_t s);
// n_res bounds the residues of every gene read through gene_ptr (genes read
// through gene_src are trusted).
cudaError_t run_encode_mark(Launcher* L, const uint8_t* res, const int64_t* gene_ptr, uint32_t n_genes, int k,
                            uint32_t* dict, const uint16_t* gene_genome,
                            const unsigned long long* genome_code_base, const int64_t* gene_src, int alpha,
                            uint64_t n_res, DevErr* err, cudaStream_t s);
// Outputs of the multiplicity-vector build.
struct MvOut {
  uint32_t* mv_id;
  uint16_t* mv_cnt;
  uint32_t* mv_n;
  unsigned long long* rec;  // [W] (id << 32) | packed posting; all-ones in unused slots
  uint32_t* minhash;
  uint32_t cnt_bits, cnt_cap;
  DevErr* err;
  const uint16_t* gene_genome;                 // genome of each gene
  const unsigned long long* genome_code_base;  // per genome: segment * 20^k, or null (one segment)
  const int64_t* gene_src;                     // per gene: first residue, or null (gene_ptr[g])
  int alpha;                                   // alphabet size: 20 or 4
  int length_buckets;                          // query order: length buckets first (1) or min-hash only (0)
  int frozen;                                  // 1: the dictionary is another dataset's; windows
                                               // whose code it lacks are left out of the vector
};
// Table slots used for a gene with La windows (genes above 16384 slots use
// global scratch of that many 64-bit slots, listed in long_genes).
uint32_t mv_build_table_cap(uint32_t La);
cudaError_t run_mv_build(Launcher* L, const uint8_t* res, const int64_t* gene_ptr, const uint32_t* win_off,
                         uint32_t n_genes, int k, const uint32_t* dict, const MvOut& M, const uint32_t* mid_genes, uint32_t n_mid, const uint32_t* long_genes,
                         uint32_t n_long, unsigned long long* long_scratch, const unsigned long long* long_scratch_off,
                         cudaStream_t s);
// Stable LSD radix sort of the n index records in `a` (ping-pong with `b`) by
// the low key_bits bits of their high word, then postings and id offsets:
// post[0..E) and post_ptr[0..n_ids] (post_ptr[n_ids] = E).  `counts` holds
// radix_counts_words(n) words; scan_tmp serves a scan of that many.
size_t radix_counts_words(uint64_t n);
cudaError_t run_index_sort(Launcher* L, unsigned long long* a, unsigned long long* b, uint64_t n, uint32_t key_bits,
                           uint32_t* counts, void* scan_tmp, uint64_t n_ids, uint32_t* post, uint32_t* post_ptr,
                           cudaStream_t s);
// Posting range of every multiplicity-vector entry; also the longest list and
// (join not null) the sum of the entries' list lengths.
cudaError_t run_mv_post(Launcher* L, const uint32_t* win_off, const uint32_t* mv_n, const uint32_t* mv_id,
                        uint32_t n_genes, const uint32_t* post_ptr, uint32_t* mv_post, uint32_t* mv_plen,
                        uint32_t* max_posting, unsigned long long* join, cudaStream_t s);
// count must hold 2 * 2^(32-shift) + 1 words (counts, then their prefix sum).
cudaError_t run_order(Launcher* L, const uint32_t* minhash, uint32_t n_genes, uint32_t shift, uint32_t* count,
                      uint32_t* order, void* scan_tmp, cudaStream_t s);
cudaError_t run_gene_info(Launcher* L, const int32_t* genome_ptr, uint32_t n_genomes, const uint32_t* La,
                          uint16_t* gene_genome, uint32_t* ginfo, cudaStream_t s);
cudaError_t run_select_codes(Launcher* L, const uint32_t* dict, uint64_t n_blocks, unsigned long long* code_of_id,
                             cudaStream_t s);
// pad_off: n_genes+1 offsets of power-of-two padded per-gene scratch regions in pad.
cudaError_t run_export_mv(Launcher* L, const ProfilesView& P, const unsigned long long* mv_ptr,
                          const unsigned long long* pad_off, unsigned long long* pad,
                          const unsigned long long* code_of_id, unsigned long long* codes, uint32_t* counts,
                          cudaStream_t s);
cudaError_t run_export_index(Launcher* L, const ProfilesView& P, int32_t* genes, uint32_t* counts,
                             cudaStream_t s);

// sum-min and Best Hits (k_summin.cu): shared-memory tiers 1 and 2 in one
// call (tier 2 reads tier 1's deferred list on the device), then, only if
// tier 2 deferred queries, the global-memory tier.
cudaError_t run_summin_tiers(Launcher* L, const ProfilesView& P, const QuerySet& Q, const HitsOut& O, DevErr* err,
                             bool emit_all, cudaStream_t s);
size_t summin_global_smem_bytes(uint32_t n_genomes);
cudaError_t run_summin_global(Launcher* L, const ProfilesView& P, const QuerySet& Q, const HitsOut& O,
                              const BigScratch& B, uint32_t n_ctas, DevErr* err, bool emit_all, cudaStream_t s);

// Symmetric all-pairs form (k_sym.cu): rows = the reverse part (from symbest
// and the valid ties, ascending) followed by the forward part of the launch.
struct SymRows {
  uint32_t n_genes, n_genomes;
  const uint16_t* gene_genome;
  const uint32_t* La;
  const unsigned long long* symbest;  // [n_genomes * n_genes], genome-major: b over genome g at g * n_genes + b
  const unsigned long long* tie_rec;  // [2 * n_ties]: (b << 32 | a), s
  unsigned long long n_ties;
  unsigned long long* tie_set;        // [tie_set_mask + 1] all-ones: the pairs already counted
  unsigned long long tie_set_mask;
  const unsigned long long* fwd_off;  // forward rows of the launch
  const uint32_t* fwd_len;
  const uint32_t* fwd_b;
  const uint32_t* fwd_s;
};
// Per gene: stored maxima (stored), valid ties (tiecnt, must start at zero;
// tie_ok flags each tie) and the row length (total).
cudaError_t run_sym_count(Launcher* L, const SymRows& R, uint32_t* stored, uint32_t* tiecnt, uint8_t* tie_ok,
                          uint32_t* total, cudaStream_t s);
// Rows written at row_ptr (exclusive scan of total); tie_fill must start at zero.
cudaError_t run_sym_write(Launcher* L, const SymRows& R, const uint32_t* stored, const uint32_t* tiecnt,
                          const uint8_t* tie_ok, const unsigned long long* row_ptr, uint32_t* tie_fill,
                          uint32_t* out_b, uint32_t* out_s, cudaStream_t s);

// BBH of the symmetric form: a forward hit is a BBH when its ratio equals the
// target's stored maximum over the query genome.  count: flags per forward
// hit, per-row counts and their exclusive scan (start[n_genes] = pairs);
// write: the pairs (a, b) ascending.
cudaError_t run_sym_bbh_count(Launcher* L, const SymRows& R, uint8_t* flag, uint32_t* cnt, uint32_t* start,
                              void* scan_tmp, cudaStream_t s);
cudaError_t run_sym_bbh_write(Launcher* L, const SymRows& R, const uint8_t* flag, const uint32_t* start, int32_t* pa,
                              int32_t* pb, cudaStream_t s);

// BBH and result gathering (k_bbh.cu)
cudaError_t run_gather_rows(Launcher* L, uint32_t n_rows, const unsigned long long* row_off,
                            const uint32_t* row_len, const unsigned long long* row_ptr, const uint32_t* in_b,
                            const uint32_t* in_s, uint32_t col_base, int32_t* out_cols, uint32_t* out_s,
                            cudaStream_t s);
// BBH from Best Hit rows.  Row x belongs to gene row_gene(x); the partner row
// of a target gene b is row_of_gene(b).  See k_bbh.cu for the two forms.
struct BbhRows {
  int all_pairs;               // 1: rows = all genes (row x = gene x)
  int paralog;                 // with all_pairs: hits inside one genome, pairs (a, b) with a < b
  uint32_t n_rows;
  uint32_t nA, qa0, qb0;       // pair form: rows 0..nA-1 = genes qa0.., rest = genes qb0..
  const uint16_t* gene_genome; // all form: genome of each gene
  const int32_t* genome_ptr;   // all form: first gene of each genome (n_genomes + 1)
  const unsigned long long* row_off;
  const uint32_t* row_len;
  const uint32_t* hit_b;
};
cudaError_t run_bbh_count(Launcher* L, const BbhRows& R, uint8_t* flags_by_hit, uint32_t* row_cnt,
                          cudaStream_t s);
cudaError_t run_bbh_write(Launcher* L, const BbhRows& R, const uint8_t* flags_by_hit, const uint32_t* row_start,
                          uint32_t a_base, uint32_t b_base, int32_t* out_a, int32_t* out_b, cudaStream_t s);

// ---------------------------------------------------------------- handle access
// Implemented in pd_api.cu; used by entry points in other files.
struct CtxView {
  cudaStream_t stream;
  int device;
  DevErr* d_err;  // device error block
  DevErr* h_err;  // its pinned host mirror
  Launcher* launcher;
};
bool ctx_view(pd_ctx* c, CtxView* v);
bool ctx_swap_timing(pd_ctx* c, bool on);  // returns the previous setting
pd_status ctx_fail(pd_ctx* c, pd_status st, const char* msg);
const ProfilesView* profiles_view(const pd_profiles* P);
int32_t profiles_genome_start(const pd_profiles* P, uint32_t g);  // genome_ptr[g] (host copy)

}  // namespace pdg
