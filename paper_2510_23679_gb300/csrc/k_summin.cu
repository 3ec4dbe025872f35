// k_summin.cu -- sum-min by inverted-index scatter, fused with Best Hit
// selection ("Best Hit detection phase", Algorithm 2, Eqs. (5) and (8)).
//
// One thread block owns one query gene a at a time:
//   1. stage a chunk of a's multiplicity vector in shared memory: for each
//      k-mer its multiplicity and posting range (stored with the vector, so
//      this read is coalesced; in the pair forms the range is narrowed by
//      binary search to the target genome, in the symmetric all-pairs form to
//      the genomes after a's own), and a block prefix sum of the range
//      lengths: the chunk's postings form one flat index space;
//   2. walk the postings, one of two ways chosen per launch: the merge-path
//      walk (thread t takes the flat range [t*P, (t+1)*P), finds its first
//      k-mer by one binary search and advances sequentially, four postings
//      loaded before any is used) or the warp-cooperative walk (each warp
//      reads 32 consecutive flat positions per round, the k-mer of each lane
//      found from the staged list starts by a warp OR-reduction); each
//      posting (b, mult_b) adds min(mult_a, mult_b) to b's accumulator in
//      shared memory: an open-addressing hash, or direct slots when the
//      query's targets are one gene range that fits the table.  After all
//      chunks acc[b] = s(a, b), the Eq. (5) numerator, exactly;
//   3. Best Hits: per target genome the maximum ratio s / (La + Lb - s) is
//      kept as an (s, den) pair updated by compare-and-swap under a 64-bit
//      cross-multiplication order; every accumulator whose ratio equals its
//      genome's maximum (again by cross-multiplication) is a Best Hit (Eq. (8),
//      ties kept).  The second pass also clears the slots it reads, so the
//      table is clean for the next query.  Each hit is written at its rank
//      among the query's hits (ascending gene): rows come out sorted without a
//      sorting network.
// In the symmetric all-pairs form each candidate b also keeps, in global
// memory, its best ratio over a's genome (the column maximum of Algorithm 3,
// with exact ties listed), from which k_sym.cu assembles the reverse rows.
// Served queries (new genomes against a resident set) may limit the targets
// to genes below a bound, and may also keep each target's best ratio over the
// query's genome in global memory (the reverse-direction maximum needed for
// the mutual check of Eq. (9)).
// The similarity matrix S_ij is never materialised: only pairs sharing a
// k-mer are touched.  A query whose insertions probe too far (a nearly full
// table), or whose Best Hit list does not fit, is deferred to the next tier:
// 4096 slots in shared memory (256 threads) -> 16384 slots in shared memory
// (1024 threads, one block per SM) -> a global-memory table sized for every
// possible target.  Results are exact and independent of the tier.
#include <algorithm>

#include "pd_internal.cuh"

namespace pdg {
namespace {

struct Scalars {
  uint32_t n_out;
  uint32_t overflow;
  uint32_t base_lo, base_hi;
  uint32_t warp_tmp[33];
};


// Probes allowed before a query counts as overflowing its table.  Long chains
// mean a nearly full table; the query then moves to a larger tier, so the
// bound never changes a result, only where it is computed.
constexpr uint32_t kMaxProbe = 64;

// Two table layouts share the code below.
//   packed (tier 1): one word per slot, (b << cnt_bits) | s.  A posting is
//     packed the same way, so the walk keys the table with the posting's own
//     high bits ("bkey") and never unpacks the gene id.  Valid while s stays
//     below the all-ones count, which holds for every query with
//     La < 2^cnt_bits - 1 (s <= La); other queries go to tier 2.  The gene
//     field never holds all ones (that id is reserved), so the empty word
//     0xFFFFFFFF matches no key.
//   split (tiers 2 and 3): keys[] = b, vals[] = s.
// Slots are found by multiplicative hashing (top bits of key * odd constant)
// and linear probing.
template <bool kPacked, bool kFilter = false>
struct Acc {
  static_assert(!(kPacked && kFilter), "filtered queries use the split layout");
  uint32_t* keys;  // packed: slot words
  uint32_t* vals;  // split only
  uint32_t* vpa;   // filtered only: sum of mult_a over the shared k-mers (Eq. (7) numerator, a -> b)
  uint32_t* vpb;   // filtered only: sum of mult_b over the shared k-mers (b -> a)
  uint32_t cnt_bits;
  uint32_t hash_shift;  // 32 - log2(cap)
  // Target genes [dense_lo, dense_lo + cap) of a query whose targets fit the
  // table: slot = gene - dense_lo (direct, the first probe always lands);
  // kEmpty: hashed slots.
  uint32_t dense_lo;

  __device__ __forceinline__ void bump(uint32_t h, uint32_t m, uint32_t ca, uint32_t cb) const {
    atomicAdd(&vals[h], m);
    if (kFilter) {
      atomicAdd(&vpa[h], ca);
      atomicAdd(&vpb[h], cb);
    }
  }

  __device__ __forceinline__ uint32_t home(uint32_t key) const {
    if (dense_lo != kEmpty) return (kPacked ? key >> cnt_bits : key) - dense_lo;
    return (key * 0x9E3779B1u) >> hash_shift;
  }

  // key: bkey (packed) or b (split).  Returns false after kMaxProbe probes.
  // ca, cb (the two multiplicities) feed the directional sums of filtered queries.
  __device__ __forceinline__ bool add(uint32_t mask, uint32_t key, uint32_t m, uint32_t ca = 0,
                                      uint32_t cb = 0) const {
    uint32_t h = home(key);
    const uint32_t hi = ~((1u << cnt_bits) - 1u);
    for (uint32_t probe = 0; probe < kMaxProbe; ++probe) {
      const uint32_t k = *((volatile uint32_t*)&keys[h]);
      if (kPacked) {
        if ((k & hi) == key) {
          atomicAdd(&keys[h], m);
          return true;
        }
        if (k == kEmpty) {
          const uint32_t prev = atomicCAS(&keys[h], kEmpty, key | m);
          if (prev == kEmpty) return true;
          if ((prev & hi) == key) {
            atomicAdd(&keys[h], m);
            return true;
          }
        }
      } else {
        if (k == key) {
          bump(h, m, ca, cb);
          return true;
        }
        if (k == kEmpty) {
          const uint32_t prev = atomicCAS(&keys[h], kEmpty, key);
          if (prev == kEmpty || prev == key) {
            bump(h, m, ca, cb);
            return true;
          }
        }
      }
      h = (h + 1) & mask;
    }
    return false;
  }
  __device__ __forceinline__ bool occupied(uint32_t h) const { return keys[h] != kEmpty; }
  __device__ __forceinline__ void get(uint32_t h, uint32_t* b, uint32_t* s) const {
    const uint32_t k = keys[h];
    if (kPacked) {
      *b = k >> cnt_bits;
      *s = k & ((1u << cnt_bits) - 1u);
    } else {
      *b = k;
      *s = vals[h];
    }
  }
  __device__ __forceinline__ void clear(uint32_t h) const {
    keys[h] = kEmpty;
    if (!kPacked) vals[h] = 0;
    if (kFilter) {
      vpa[h] = 0;
      vpb[h] = 0;
    }
  }
};

// Eqs. (6) and (7) as candidate masks: lengths |g| = La + k - 1 (a candidate
// shares a k-mer, so La >= 1 on both sides), directional sums against La.
__device__ __forceinline__ bool filter_pass(const QuerySet& Q, uint32_t k, uint32_t La_a, uint32_t La_b, uint32_t pa,
                                            uint32_t pb) {
  if (Q.theta_num) {
    const unsigned long long la = La_a + k - 1u, lb = La_b + k - 1u;
    if (la * Q.theta_den < (unsigned long long)Q.theta_num * lb) return false;
    if (lb * Q.theta_den < (unsigned long long)Q.theta_num * la) return false;
  }
  if (Q.tau_num) {
    if ((unsigned long long)pa * Q.tau_den < (unsigned long long)Q.tau_num * La_a) return false;
    if ((unsigned long long)pb * Q.tau_den < (unsigned long long)Q.tau_num * La_b) return false;
  }
  return true;
}

__device__ __forceinline__ uint32_t lower_bound_post(const uint32_t* __restrict__ post, uint32_t lo, uint32_t hi,
                                                     unsigned long long key) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if ((unsigned long long)post[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Exact multiplicity of k-mer id in gene g, for a saturated packed count.
// A multiplicity vector is stored in hash order, so this is a linear scan
// (rare: only counts at the cap of the packed field come here).
__device__ __forceinline__ uint32_t mv_count_of(const ProfilesView& P, uint32_t g, uint32_t id) {
  const uint32_t off = P.win_off[g], n = P.mv_n[g];
  for (uint32_t e = 0; e < n; ++e)
    if (P.mv_id[off + e] == id) return P.mv_cnt[off + e];
  return 0u;
}

// Max of (s, den) pairs by cross-multiplication, packed as s << 32 | den.
__device__ __forceinline__ void best_update(unsigned long long* slot, uint32_t s, uint32_t den) {
  unsigned long long old = *((volatile unsigned long long*)slot);
  const unsigned long long mine = ((unsigned long long)s << 32) | den;
  while (true) {
    const uint32_t os = (uint32_t)(old >> 32), od = (uint32_t)old;
    if (os != 0 && !ratio_greater(s, den, os, od)) return;
    const unsigned long long prev = atomicCAS(slot, old, mine);
    if (prev == old) return;
    old = prev;
  }
}

// Reverse-direction maximum of the symmetric form: the best (s, den) of
// target b over the query genome, with the query gene a that reaches it,
// packed s << 48 | den << 31 | a (s < 2^16, den < 2^17, a < 2^31); a pair
// that equals the stored maximum is listed as a tie (b << 32 | a, s).  Ties of
// a maximum later beaten stay in the list and are dropped when the rows are
// assembled.
__device__ __forceinline__ void sym_update(const QuerySet& Q, unsigned long long* slot, uint32_t b, uint32_t a,
                                           uint32_t s, uint32_t den) {
  const unsigned long long mine =
      ((unsigned long long)s << 48) | ((unsigned long long)den << 31) | (unsigned long long)a;
  unsigned long long old = *((volatile unsigned long long*)slot);
  while (true) {
    if (old != 0ull) {
      const uint32_t os = (uint32_t)(old >> 48), od = (uint32_t)(old >> 31) & 0x1FFFFu;
      if (ratio_greater(os, od, s, den)) return;
      if (ratio_equal(os, od, s, den)) {
        const unsigned long long t = atomicAdd(Q.tie_count, 1ull);
        if (t < Q.tie_cap) {
          Q.tie_rec[2 * t] = ((unsigned long long)b << 32) | a;
          Q.tie_rec[2 * t + 1] = s;
        }
        return;
      }
    }
    const unsigned long long prev = atomicCAS(slot, old, mine);
    if (prev == old) return;
    old = prev;
  }
}

template <int kThreads>
struct Chunk {
  static constexpr uint32_t kSize = 2 * kThreads;  // query k-mers staged per round
  static constexpr uint32_t kItems = 2;
  // c_post (4 B), c_off (4 B, one more), c_cnt (2 B), c_ent (2 B) per k-mer
  static constexpr size_t kBytes =
      (((size_t)kSize * 4 + (size_t)(kSize + 1) * 4 + (size_t)kSize * 2 + (size_t)kSize * 2) + 15) & ~(size_t)15;
};

// Rounds of 32 postings a warp has in flight before accumulating them (the
// warp-cooperative walk), and the average posting-list length, weighted by
// use (a dataset's join over its vector entries), from which tier 1 takes
// that walk rather than the merge-path walk: a warp round then reads few
// lists, while for short lists each thread's run of postings stays within the
// sectors it has already loaded.
constexpr uint32_t kRounds = 4;
constexpr uint32_t kWarpWalkMinAvg = 16;
// ... and the smallest index (4-byte postings) for which the warp walk is
// taken: below a few L2 sizes the merge-path walk's runs of postings keep
// hitting the sectors they have already brought in.
constexpr uint64_t kWarpWalkMinIndexBytes = 512ull << 20;
// Target genomes from which a query's Best Hits are ranked through per-genome
// positions rather than pairwise.
constexpr uint32_t kRankByGenomeMin = 64;

// Memory of one call: table, the list of occupied slots (filled after the
// walk) and the hit list.
template <typename TIdx>
struct Table {
  uint32_t* keys;
  uint32_t* vals;          // split layout only
  uint32_t* vpa;           // filtered queries only
  uint32_t* vpb;
  TIdx* used;              // capacity used_cap
  unsigned long long* out; // capacity out_cap
  uint32_t cap;            // power of two, a multiple of the block size
  uint32_t out_cap;
  uint32_t used_cap;       // at most cap; a query with more occupied slots moves to the next tier
};

template <int kThreads, bool kEmitAll, bool kPacked, bool kFilter, typename TIdx, bool kWarpWalk>
__device__ __forceinline__ void process_query(uint32_t qi, const ProfilesView& P, const QuerySet& Q,
                                              const HitsOut& O, const TierIO& T, DevErr* err,
                                              const Table<TIdx>& tb, uint32_t* c_post, uint32_t* c_off,
                                              uint16_t* c_cnt, unsigned long long* best, Scalars* sh) {
  constexpr uint32_t kChunk = Chunk<kThreads>::kSize, kItems = Chunk<kThreads>::kItems;
  Acc<kPacked, kFilter> acc{tb.keys, tb.vals, tb.vpa, tb.vpb, P.cnt_bits, 32u - (31u - (uint32_t)__clz(tb.cap)), kEmpty};
  uint16_t* c_ent = c_cnt + Chunk<kThreads>::kSize;  // chunk entry of each staged k-mer
  unsigned long long* out = tb.out;
  const uint32_t mask = tb.cap - 1u;
  // ---- query gene, its output row and its targets
  uint32_t a, row, own0 = 0, own1 = 0, tend = 0xFFFFFFFFu, col = 0, self = kEmpty;
  unsigned long long key_lo = 0, key_hi = 0;
  if (Q.all_pairs) {
    a = Q.order ? Q.order[qi] : Q.q0 + qi;
    if (Q.n_shards && a % Q.n_shards != Q.shard) return;  // another shard's query (uniform over the block)
    row = a;
    if (Q.q_genome) {  // external query: no own genome among the targets
      const uint32_t x = Q.q_genome[a];
      own0 = own1 = kEmpty;
      if (Q.tgt_end) tend = Q.tgt_end[x];
      col = x;
    } else {
      const uint32_t gg = P.gene_genome[a];
      own0 = (uint32_t)P.genome_ptr[gg];
      own1 = (uint32_t)P.genome_ptr[gg + 1];
      if (Q.tgt_end) tend = Q.tgt_end[gg];
      col = gg - Q.col_genome0;
      if (Q.symbest) key_lo = (unsigned long long)own1 << P.cnt_bits;  // first posting past a's genome
    }
  } else {
    uint32_t tlo, thi;
    if (Q.q_gene) {
      a = Q.q_gene[qi];
      tlo = Q.q_t0[qi];
      thi = Q.q_t1[qi];
    } else if (Q.paralog) {
      a = Q.q0 + qi;
      const uint32_t gg = P.gene_genome[a];
      tlo = (uint32_t)P.genome_ptr[gg];
      thi = (uint32_t)P.genome_ptr[gg + 1];
      self = a;
    } else if (qi < Q.nA) {
      a = Q.qa0 + qi;
      tlo = Q.ta0;
      thi = Q.ta1;
    } else {
      a = Q.qb0 + (qi - Q.nA);
      tlo = Q.tb0;
      thi = Q.tb1;
    }
    row = qi;
    key_lo = (unsigned long long)tlo << P.cnt_bits;
    key_hi = (unsigned long long)thi << P.cnt_bits;
  }
  // one target range that fits the table: direct slots instead of hashing
  if (!Q.all_pairs) {
    const uint32_t tlo = (uint32_t)(key_lo >> P.cnt_bits), thi = (uint32_t)(key_hi >> P.cnt_bits);
    if (thi > tlo && thi - tlo <= tb.cap) acc.dense_lo = tlo;
  }
  // the query's own vector (its dataset's, or the external query arrays)
  const bool ext = P.q_win_off != nullptr;
  const uint32_t* __restrict__ q_mv_id = ext ? P.q_mv_id : P.mv_id;
  const uint16_t* __restrict__ q_mv_cnt = ext ? P.q_mv_cnt : P.mv_cnt;
  const uint32_t* __restrict__ q_mv_post = ext ? P.q_mv_post : P.mv_post;
  const uint32_t* __restrict__ q_mv_plen = ext ? P.q_mv_plen : P.mv_plen;
  const uint32_t m0 = (ext ? P.q_win_off : P.win_off)[a], E = (ext ? P.q_mv_n : P.mv_n)[a];
  const uint32_t La_a = (ext ? P.q_La : P.La)[a];
  const uint32_t cnt_mask = (1u << P.cnt_bits) - 1u;
  const uint32_t tid = threadIdx.x;
  if (tid == 0) {
    sh->n_out = 0;
    // a packed slot holds s <= La_a: queries beyond the field go to tier 2
    sh->overflow = (kPacked && La_a >= cnt_mask) ? 1u : 0u;
  }
  __syncthreads();
  unsigned long long walked = 0;
  const uint32_t lane = tid & 31u, warp = tid >> 5;
  constexpr uint32_t kWarps = kThreads / 32;
  for (uint32_t c0 = 0; c0 < E && !sh->overflow; c0 += kChunk) {
    const uint32_t n_in = min(kChunk, E - c0);
    // Each posting (b, mult_b) adds min(mult_a, mult_b) to b's accumulator.
    // Own-genome postings are accumulated too and dropped when the Best Hits
    // are chosen (a few slots per query), which keeps the walks free of
    // per-posting range tests.  `e` is the query's chunk entry of the k-mer.
    auto accumulate = [&](uint32_t p, uint32_t ca, uint32_t e) {
      uint32_t cb = p & cnt_mask;
      if (cb == P.cnt_cap && ca > cb) cb = mv_count_of(P, p >> P.cnt_bits, q_mv_id[m0 + c0 + e]);
      const uint32_t key = kPacked ? (p & ~cnt_mask) : (p >> P.cnt_bits);
      if (!acc.add(mask, key, min(ca, cb), ca, cb)) sh->overflow = 1;
    };
    if constexpr (kWarpWalk) {
      // ---- stage the chunk: posting ranges and their prefix sum.  Empty
      // ranges (the restricted forms narrow lists to a target genome) are
      // dropped, so the staged list starts strictly increase, as the walk's
      // k-mer lookup needs.
      uint32_t lo_loc[kItems], len_loc[kItems];
      uint32_t my_sum = 0, my_n = 0;
#pragma unroll
      for (uint32_t r = 0; r < kItems; ++r) {
        const uint32_t e = tid * kItems + r;
        uint32_t lo = 0, len = 0;
        if (e < n_in) {
          lo = q_mv_post[m0 + c0 + e];
          const uint32_t plen = q_mv_plen[m0 + c0 + e];
          uint32_t hi = lo + plen;
          if (!ext && plen == 1u) {
            hi = lo;  // the list holds only the query's own posting: never a target
          } else if (!Q.all_pairs) {
            lo = lower_bound_post(P.post, lo, hi, key_lo);
            hi = lower_bound_post(P.post, lo, hi, key_hi);
          } else if (Q.symbest) {
            lo = lower_bound_post(P.post, lo, hi, key_lo);  // the genomes after the query's own
          }
          len = hi - lo;
        }
        lo_loc[r] = lo;
        len_loc[r] = len;
        my_sum += len;
        my_n += len ? 1u : 0u;
      }
      uint32_t J_c, n_c;
      uint32_t run = block_exclusive_scan(my_sum, sh->warp_tmp, &J_c);
      uint32_t slot = block_exclusive_scan(my_n, sh->warp_tmp, &n_c);
#pragma unroll
      for (uint32_t r = 0; r < kItems; ++r) {
        const uint32_t e = tid * kItems + r;
        if (len_loc[r]) {
          c_post[slot] = lo_loc[r];
          c_cnt[slot] = q_mv_cnt[m0 + c0 + e];
          c_ent[slot] = (uint16_t)e;
          c_off[slot] = run;
          ++slot;
        }
        run += len_loc[r];
      }
      if (tid == 0) c_off[n_c] = J_c;
      __syncthreads();
      walked += J_c;
      // ---- warp-cooperative walk.  Warp w takes the flat postings [x0, x1)
      // and reads them 32 consecutive positions per round, lane l position
      // xr + l, so a round reads one or a few lists contiguously.  The k-mer
      // of each lane's position comes from the starts of the next 32 staged
      // k-mers (one per lane): bit d of `starts` marks a k-mer starting d
      // positions after the round's first, and a lane's k-mer is the round's
      // first k-mer plus the number of starts at or before it.
      const uint32_t per_w = ((J_c + kWarps - 1) / kWarps + 31u) & ~31u;
      const uint32_t x0 = min(J_c, warp * per_w), x1 = min(J_c, x0 + per_w);
      if (x0 < x1) {
        uint32_t e_lo = 0, hi = n_c;  // the k-mer holding x0: last e with c_off[e] <= x0
        while (hi - e_lo > 1) {
          const uint32_t mid = (e_lo + hi) >> 1;
          if (c_off[mid] <= x0) e_lo = mid; else hi = mid;
        }
        for (uint32_t xb = x0; xb < x1; xb += 32u * kRounds) {
          uint32_t pv[kRounds], cav[kRounds], ev[kRounds];
#pragma unroll
          for (uint32_t u = 0; u < kRounds; ++u) {
            const uint32_t xr = xb + 32u * u, x = xr + lane;
            const uint32_t j = e_lo + 1u + lane;
            const uint32_t d = (j <= n_c && xr < x1) ? c_off[j] - xr : 0xFFFFFFFFu;
            const uint32_t starts = __reduce_or_sync(0xFFFFFFFFu, d < 32u ? (1u << d) : 0u);
            const uint32_t e = e_lo + __popc(starts & (0xFFFFFFFFu >> (31u - lane)));
            e_lo += __popc(starts) + (__ballot_sync(0xFFFFFFFFu, d == 32u) ? 1u : 0u);
            pv[u] = kEmpty;
            cav[u] = 0;
            ev[u] = 0;
            if (x < x1) {
              pv[u] = P.post[c_post[e] + (x - c_off[e])];
              cav[u] = c_cnt[e];
              ev[u] = c_ent[e];
            }
          }
#pragma unroll
          for (uint32_t u = 0; u < kRounds; ++u)
            if (xb + 32u * u + lane < x1) accumulate(pv[u], cav[u], ev[u]);
        }
      }
    } else {
      // ---- stage the chunk: posting ranges and their prefix sum
      uint32_t len_loc[kItems];
      uint32_t my_sum = 0;
#pragma unroll
      for (uint32_t r = 0; r < kItems; ++r) {
        const uint32_t e = tid * kItems + r;
        uint32_t len = 0;
        if (e < n_in) {
          uint32_t lo = q_mv_post[m0 + c0 + e];
          uint32_t hi = lo + q_mv_plen[m0 + c0 + e];
          if (!Q.all_pairs) {
            lo = lower_bound_post(P.post, lo, hi, key_lo);
            hi = lower_bound_post(P.post, lo, hi, key_hi);
          } else if (Q.symbest) {
            lo = lower_bound_post(P.post, lo, hi, key_lo);  // the genomes after the query's own
          }
          c_post[e] = lo;
          c_cnt[e] = q_mv_cnt[m0 + c0 + e];
          len = hi - lo;
        }
        len_loc[r] = len;
        my_sum += len;
      }
      uint32_t J_c;
      uint32_t run = block_exclusive_scan(my_sum, sh->warp_tmp, &J_c);
#pragma unroll
      for (uint32_t r = 0; r < kItems; ++r) {
        const uint32_t e = tid * kItems + r;
        if (e < n_in) c_off[e] = run;
        run += len_loc[r];
      }
      if (tid == 0) c_off[n_in] = J_c;
      __syncthreads();
      walked += J_c;
      // ---- merge-path walk: thread t takes the flat range [t*per,
      // (t+1)*per), finds its first k-mer by one binary search and then
      // advances sequentially, loading four postings before using any (a
      // thread's next postings mostly share the sector of its last one).
      const uint32_t per = (J_c + kThreads - 1) / kThreads;
      uint32_t x = min(J_c, tid * per);
      const uint32_t x_end = min(J_c, x + per);
      if (x < x_end) {
        uint32_t lo = 0, hi = n_in;
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (c_off[mid] <= x) lo = mid; else hi = mid;
        }
        uint32_t e = lo, e_end = c_off[lo + 1], base = c_post[lo] - c_off[lo], ca = c_cnt[lo];
        while (x < x_end) {
          uint32_t pv[4], cav[4], ev[4];
          uint32_t nb = 0;
#pragma unroll
          for (uint32_t j = 0; j < 4; ++j) {
            if (x < x_end) {
              while (x >= e_end) {
                ++e;
                e_end = c_off[e + 1];
                base = c_post[e] - c_off[e];
                ca = c_cnt[e];
              }
              pv[j] = P.post[base + x];
              cav[j] = ca;
              ev[j] = e;
              ++x;
              nb = j + 1;
            }
          }
#pragma unroll
          for (uint32_t j = 0; j < 4; ++j)
            if (j < nb) accumulate(pv[j], cav[j], ev[j]);
        }
      }
    }
    __syncthreads();
  }

  bool overflow = sh->overflow != 0;
  const uint32_t n_best = Q.all_pairs ? P.n_genomes : 1u;
  // With few target genomes a row has few hits and ranking them pairwise is
  // cheaper than a block scan over the genomes.
  const bool by_genome = !kEmitAll && n_best >= kRankByGenomeMin;
  // Best Hits of each target genome, then (exclusive scan) the first output
  // position of each genome's hits: rows come out ordered by gene because
  // genes are numbered genome by genome
  uint32_t* hcnt = (uint32_t*)(best + n_best);
  // Slots are visited interleaved (slot = i * kThreads + tid: conflict-free).
  const uint32_t slots = tb.cap / kThreads;
  uint32_t n_occ = 0, pos = 0;
  if (!overflow) {
    // ---- count the occupied slots (block prefix sum over per-thread counts);
    // more than the list holds: the query moves to the next tier
    uint32_t n_mine = 0;
    for (uint32_t i = 0; i < slots; ++i) n_mine += acc.occupied(i * kThreads + tid) ? 1u : 0u;
    pos = block_exclusive_scan(n_mine, sh->warp_tmp, &n_occ);
    overflow = n_occ > tb.used_cap;  // uniform over the block
  }
  if (!overflow) {
    // ---- list them
    for (uint32_t i = 0; i < slots; ++i) {
      const uint32_t h = i * kThreads + tid;
      if (acc.occupied(h)) tb.used[pos++] = (TIdx)h;
    }
    __syncthreads();
    if (kEmitAll) {
      for (uint32_t u = tid; u < n_occ; u += kThreads) {
        const uint32_t h = tb.used[u];
        uint32_t b, s;
        acc.get(h, &b, &s);
        const uint32_t slot = atomicAdd(&sh->n_out, 1u);
        if (slot < tb.out_cap) out[slot] = ((unsigned long long)b << 32) | s;
        acc.clear(h);
      }
    } else {
      // ---- per target genome: the maximum ratio, then every entry at it
      for (uint32_t j = tid; j < n_best; j += kThreads) {
        best[j] = 0ull;
        if (by_genome) hcnt[j] = 0u;
      }
      __syncthreads();
      for (uint32_t u = tid; u < n_occ; u += kThreads) {
        uint32_t b, s;
        acc.get(tb.used[u], &b, &s);
        if ((Q.all_pairs && ((b >= own0 && b < own1) || b >= tend)) || b == self) continue;  // not a target
        const uint32_t gi = P.ginfo[b];
        if (kFilter && !filter_pass(Q, P.k, La_a, gi & 0xFFFFu, acc.vpa[tb.used[u]], acc.vpb[tb.used[u]])) continue;
        const uint32_t den = La_a + (gi & 0xFFFFu) - s;
        best_update(&best[Q.all_pairs ? (gi >> 16) : 0u], s, den);
        if (Q.colbest) best_update(&Q.colbest[(size_t)b * Q.col_stride + col], s, den);
        if (Q.symbest) sym_update(Q, &Q.symbest[(size_t)col * P.n_genes + b], b, a, s, den);
      }
      __syncthreads();
      for (uint32_t u = tid; u < n_occ; u += kThreads) {
        const uint32_t h = tb.used[u];
        uint32_t b, s;
        acc.get(h, &b, &s);
        const uint32_t gi = P.ginfo[b];
        const unsigned long long bv = best[Q.all_pairs ? (gi >> 16) : 0u];
        if (!(Q.all_pairs && ((b >= own0 && b < own1) || b >= tend)) && b != self &&
            (!kFilter || filter_pass(Q, P.k, La_a, gi & 0xFFFFu, acc.vpa[h], acc.vpb[h])) &&
            ratio_equal(s, La_a + (gi & 0xFFFFu) - s, (uint32_t)(bv >> 32), (uint32_t)bv)) {
          // s <= La <= 65535 and the genome < 65536: (b, genome, s) in one word
          const uint32_t g = Q.all_pairs ? (gi >> 16) : 0u;
          const uint32_t slot = atomicAdd(&sh->n_out, 1u);
          if (slot < tb.out_cap) out[slot] = ((unsigned long long)b << 32) | (g << 16) | s;
          if (by_genome) atomicAdd(&hcnt[g], 1u);
        }
        acc.clear(h);
      }
    }
  } else {
    // the walk stopped early, or the occupied slots do not fit the list: clear every slot
    for (uint32_t i = 0; i < slots; ++i) acc.clear(i * kThreads + tid);
  }
  __syncthreads();
  const uint32_t n_out = sh->n_out;
  if (overflow || n_out > tb.out_cap) {
    if (tid == 0) {
      if (T.def_list) {
        T.def_list[atomicAdd(T.def_count, 1u)] = qi;
      } else {
        raise_error(err, PD_ERR_INTERNAL, qi);  // the last tier holds every target
      }
      O.row_off[row] = 0;
      O.row_len[row] = 0;
    }
    __syncthreads();
    return;
  }
  if (by_genome) {
    // ---- first output position of each target genome's hits (exclusive
    // scan of the per-genome counts; each thread scans a run of genomes)
    const uint32_t per = (n_best + kThreads - 1) / kThreads;
    const uint32_t j0 = min(n_best, tid * per), j1 = min(n_best, j0 + per);
    uint32_t mine = 0;
    for (uint32_t j = j0; j < j1; ++j) mine += hcnt[j];
    uint32_t total;
    uint32_t run = block_exclusive_scan(mine, sh->warp_tmp, &total);
    for (uint32_t j = j0; j < j1; ++j) {
      const uint32_t c = hcnt[j];
      hcnt[j] = run;
      run += c;
    }
    if (tid == 0) hcnt[n_best] = total;
    __syncthreads();
  }
  // ---- append: each hit goes to its rank among the query's hits
  if (tid == 0) {
    const unsigned long long base = atomicAdd(O.cursor, (unsigned long long)n_out);
    sh->base_lo = (uint32_t)base;
    sh->base_hi = (uint32_t)(base >> 32);
    O.row_off[row] = base;
    O.row_len[row] = n_out;
    atomicAdd(O.walked, walked);
  }
  __syncthreads();
  const unsigned long long base = ((unsigned long long)sh->base_hi << 32) | sh->base_lo;
  if (base + n_out <= O.out_cap) {
    for (uint32_t t = tid; t < n_out; t += kThreads) {
      const unsigned long long v = out[t];
      const uint32_t b = (uint32_t)(v >> 32);
      uint32_t rank = 0, sv;
      if (!by_genome) {
        // rank = hits with a smaller gene id (the genome field sits below the
        // gene id, so comparing whole words orders by gene)
        for (uint32_t u = 0; u < n_out; ++u) rank += (out[u] < v) ? 1u : 0u;
        sv = kEmitAll ? (uint32_t)v : ((uint32_t)v & 0xFFFFu);
      } else {
        // the genome's first position, plus the tied hits of the same genome
        // with a smaller gene id (genomes with one Best Hit skip the loop)
        const uint32_t g = ((uint32_t)v >> 16) & 0xFFFFu;
        rank = hcnt[g];
        if (hcnt[g + 1] - rank > 1u)
          for (uint32_t u = 0; u < n_out; ++u) {
            const unsigned long long w = out[u];
            rank += ((((uint32_t)w >> 16) & 0xFFFFu) == g && (uint32_t)(w >> 32) < b) ? 1u : 0u;
          }
        sv = (uint32_t)v & 0xFFFFu;
      }
      O.out_b[base + rank] = b;
      O.out_s[base + rank] = sv;
    }
  }
  __syncthreads();
}

// ---- shared-memory tiers: [table][chunk | (used list, hits)][best]
template <int kThreads, uint32_t kCap, uint32_t kOutCap, bool kPacked, bool kFilter = false,
          uint32_t kUsedCap = kCap>
struct SmemTier {
  static_assert(kCap % kThreads == 0, "table must split evenly over the block");
  static_assert(kCap <= 65536, "slot indices are 16-bit");
  static_assert(kUsedCap <= kCap && kUsedCap % 8 == 0, "occupied-slot list");
  static constexpr size_t kTable = (size_t)kCap * (kPacked ? 4 : (kFilter ? 16 : 8));
  static constexpr size_t kUsed = (size_t)kUsedCap * 2;
  static constexpr size_t kAfterWalk = kUsed + (size_t)kOutCap * 8;
  static constexpr size_t kUnion = Chunk<kThreads>::kBytes > kAfterWalk ? Chunk<kThreads>::kBytes : kAfterWalk;
  // per target genome: best ratio (8 B) and hit count / first position (4 B), one more position
  static constexpr size_t bytes(uint32_t n_best) { return kTable + kUnion + (size_t)(n_best ? n_best : 1) * 12 + 4; }
};

template <int kThreads, int kMinBlocks, uint32_t kCap, uint32_t kOutCap, bool kPacked, bool kEmitAll,
          bool kFilter = false, uint32_t kUsedCap = kCap, bool kWarpWalk = false>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_summin_smem(ProfilesView P, QuerySet Q, HitsOut O,
                                                                      TierIO T, DevErr* err) {
  using S = SmemTier<kThreads, kCap, kOutCap, kPacked, kFilter, kUsedCap>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Scalars sh;
  Table<uint16_t> tb;
  tb.keys = (uint32_t*)smem;
  tb.vals = kPacked ? nullptr : tb.keys + kCap;
  tb.vpa = kFilter ? tb.vals + kCap : nullptr;
  tb.vpb = kFilter ? tb.vpa + kCap : nullptr;
  tb.cap = kCap;
  tb.out_cap = kOutCap;
  tb.used_cap = kUsedCap;
  unsigned char* uni = smem + S::kTable;
  tb.used = (uint16_t*)uni;
  tb.out = (unsigned long long*)(uni + S::kUsed);
  uint32_t* c_post = (uint32_t*)uni;
  uint32_t* c_off = c_post + Chunk<kThreads>::kSize;
  uint16_t* c_cnt = (uint16_t*)(c_off + Chunk<kThreads>::kSize + 1);
  unsigned long long* best = (unsigned long long*)(uni + S::kUnion);
  for (uint32_t h = threadIdx.x; h < kCap; h += kThreads) {
    tb.keys[h] = kEmpty;
    if (!kPacked) tb.vals[h] = 0;
    if (kFilter) {
      tb.vpa[h] = 0;
      tb.vpb[h] = 0;
    }
  }
  __syncthreads();
  const uint32_t n = T.in_list ? *T.in_count : Q.n_queries;
  for (uint32_t x = blockIdx.x; x < n; x += gridDim.x)
    process_query<kThreads, kEmitAll, kPacked, kFilter, uint16_t, kWarpWalk>(T.in_list ? T.in_list[x] : x, P, Q, O, T, err, tb, c_post,
                                                         c_off, c_cnt, best, &sh);
}

// ---- global-memory tier: table, used list and hit list of each block in scratch
template <bool kEmitAll, bool kFilter = false>
__global__ void __launch_bounds__(256) k_summin_global(ProfilesView P, QuerySet Q, HitsOut O, TierIO T,
                                                       BigScratch B, DevErr* err) {
  constexpr int kThreads = 256;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Scalars sh;
  Table<uint32_t> tb;
  tb.keys = B.keys + (size_t)blockIdx.x * B.cap;
  tb.vals = B.vals + (size_t)blockIdx.x * B.cap;
  tb.vpa = kFilter ? B.vpa + (size_t)blockIdx.x * B.cap : nullptr;
  tb.vpb = kFilter ? B.vpb + (size_t)blockIdx.x * B.cap : nullptr;
  tb.used = B.used + (size_t)blockIdx.x * B.cap;
  tb.out = B.out + (size_t)blockIdx.x * B.out_cap;
  tb.cap = B.cap;
  tb.out_cap = B.out_cap;
  tb.used_cap = B.cap;
  uint32_t* c_post = (uint32_t*)smem;
  uint32_t* c_off = c_post + Chunk<kThreads>::kSize;
  uint16_t* c_cnt = (uint16_t*)(c_off + Chunk<kThreads>::kSize + 1);
  unsigned long long* best = (unsigned long long*)(smem + Chunk<kThreads>::kBytes);
  for (uint32_t h = threadIdx.x; h < B.cap; h += kThreads) {
    tb.keys[h] = kEmpty;
    tb.vals[h] = 0;
    if (kFilter) {
      tb.vpa[h] = 0;
      tb.vpb[h] = 0;
    }
  }
  __syncthreads();
  const uint32_t n = *T.in_count;
  for (uint32_t x = blockIdx.x; x < n; x += gridDim.x)
    process_query<kThreads, kEmitAll, false, kFilter, uint32_t, false>(T.in_list[x], P, Q, O, T, err, tb, c_post, c_off, c_cnt, best,
                                                       &sh);
}

// Tier 1 (packed 4096-slot table, several blocks per SM) and tier 2 (split
// 16384-slot table, one 1024-thread block per SM) geometries.
constexpr int kT1Threads = 256, kT1MinBlocks = 6;
// Three tier-1 layouts, chosen per launch.  The compact one keeps six blocks
// within the 164 KB shared-memory carveout of an SM, which leaves 92 KB of
// the SM's 256 KB as L1 for the posting loads of the walk (with 4 KB more per
// block the carveout steps up to 196 KB and L1 shrinks to 60 KB): at most 3072
// listed occupied slots and 448 hits per query, a query beyond either moving
// to tier 2.  Past kT1CompactGenomes target genomes the per-genome maxima (12
// bytes each) no longer leave room for that; the middle layout lists at most
// 2048 occupied slots and 384 hits and stays within 164 KB up to
// kT1MidGenomes genomes; past that the full layout (4096 slots listed, 512
// hits) takes the 196 KB carveout.
constexpr uint32_t kT1Cap = 4096, kT1OutEmit = 3072;
constexpr uint32_t kT1Out = 448, kT1Used = 3072;          // compact layout
constexpr uint32_t kT1OutFull = 512, kT1UsedFull = 4096;  // full layout
constexpr uint32_t kT1UsedMid = 2048, kT1OutMid = 384;    // middle layout
constexpr int kT2Threads = 1024;
constexpr uint32_t kT2Cap = 16384, kT2Out = 2048, kT2OutEmit = 4096;
using T1 = SmemTier<kT1Threads, kT1Cap, kT1Out, true, false, kT1Used>;
using T1F = SmemTier<kT1Threads, kT1Cap, kT1OutFull, true, false, kT1UsedFull>;
using T1M = SmemTier<kT1Threads, kT1Cap, kT1OutMid, true, false, kT1UsedMid>;
using T1E = SmemTier<kT1Threads, kT1Cap, kT1OutEmit, true, false, kT1Used>;
// genomes up to which six compact blocks (with their static scalars and the
// 1 KB the runtime reserves per block) fit a 164 KB carveout
constexpr uint32_t kT1CompactGenomes =
    (uint32_t)((164u * 1024u / kT1MinBlocks - 1024u - sizeof(Scalars) - T1::kTable - T1::kUnion - 4u) / 12u);
static_assert(kT1CompactGenomes >= 50, "compact tier-1 layout holds tens of genomes");
// ... and six middle-layout blocks (a shorter occupied-slot list)
constexpr uint32_t kT1MidGenomes =
    (uint32_t)((164u * 1024u / kT1MinBlocks - 1024u - sizeof(Scalars) - T1M::kTable - T1M::kUnion - 4u) / 12u);
static_assert(kT1MidGenomes >= 200, "middle tier-1 layout holds hundreds of genomes");
using T2 = SmemTier<kT2Threads, kT2Cap, kT2Out, false>;
using T2E = SmemTier<kT2Threads, kT2Cap, kT2OutEmit, false>;
static_assert(T1F::bytes(PD_MAX_GENOMES) <= 227 * 1024, "tier 1 shared memory");
static_assert(T2::bytes(PD_MAX_GENOMES) <= 227 * 1024, "tier 2 shared memory");
static_assert(T2E::bytes(1) <= 227 * 1024, "tier 2 (emit-all, one target genome) shared memory");
// Filtered queries (Eqs. (6)-(7)): split 4096-slot table with the two
// directional sums; what does not fit goes straight to the global tier.
constexpr int kFThreads = 256, kFMinBlocks = 2;
constexpr uint32_t kFCap = 4096, kFOut = 512;
using TF = SmemTier<kFThreads, kFCap, kFOut, false, true>;
static_assert(TF::bytes(PD_MAX_GENOMES) <= 227 * 1024, "filtered tier shared memory");

template <typename K>
cudaError_t launch_smem(K kernel, Launcher* L, const char* name, int threads, size_t smem, uint32_t max_grid,
                        const ProfilesView& P, const QuerySet& Q, const HitsOut& O, const TierIO& T, DevErr* err,
                        cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1, dev = 0, n_sm = 152;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t grid = std::max<uint32_t>(1, std::min<uint32_t>(max_grid, (uint32_t)n_sm * std::max(per_sm, 1)));
  if ((e = launch_begin(L, name)) != cudaSuccess) return e;
  kernel<<<grid, threads, smem, s>>>(P, Q, O, T, err);
  return launch_end(L, name);
}

}  // namespace

cudaError_t run_summin_tiers(Launcher* L, const ProfilesView& P, const QuerySet& Q, const HitsOut& O, DevErr* err,
                             bool emit_all, cudaStream_t s) {
  if (Q.n_queries == 0) return cudaSuccess;
  const uint32_t n_best = Q.all_pairs ? P.n_genomes : 1u;
  if (Q.filter) {
    if (emit_all) return cudaErrorInvalidValue;
    TierIO tf{nullptr, nullptr, O.def2, O.n_def2};
    return launch_smem(k_summin_smem<kFThreads, kFMinBlocks, kFCap, kFOut, false, false, true>, L, "summin_bh_f",
                       kFThreads, TF::bytes(n_best), Q.n_queries, P, Q, O, tf, err, s);
  }
  TierIO t1{nullptr, nullptr, O.def1, O.n_def1};
  TierIO t2{O.def1, O.n_def1, O.def2, O.n_def2};
  cudaError_t e;
  // tier 1: several resident blocks per SM, each looping over queries
  if (emit_all)
    e = launch_smem(k_summin_smem<kT1Threads, kT1MinBlocks, kT1Cap, kT1OutEmit, true, true, false, kT1Used>, L, "summin_pairs",
                    kT1Threads, T1E::bytes(n_best), Q.n_queries, P, Q, O, t1, err, s);
  else if (Q.walk == PD_WALK_MERGE ||
           (Q.walk != PD_WALK_WARP && (P.n_join < (uint64_t)kWarpWalkMinAvg * P.n_entries ||
                                       P.n_entries * 4ull < kWarpWalkMinIndexBytes)))  // merge-path walk
    e = n_best <= kT1CompactGenomes
            ? launch_smem(k_summin_smem<kT1Threads, kT1MinBlocks, kT1Cap, kT1Out, true, false, false, kT1Used>, L,
                          "summin_bh", kT1Threads, T1::bytes(n_best), Q.n_queries, P, Q, O, t1, err, s)
        : n_best <= kT1MidGenomes
            ? launch_smem(k_summin_smem<kT1Threads, kT1MinBlocks, kT1Cap, kT1OutMid, true, false, false, kT1UsedMid>, L,
                          "summin_bh", kT1Threads, T1M::bytes(n_best), Q.n_queries, P, Q, O, t1, err, s)
            : launch_smem(k_summin_smem<kT1Threads, kT1MinBlocks, kT1Cap, kT1OutFull, true, false, false, kT1UsedFull>,
                          L, "summin_bh", kT1Threads, T1F::bytes(n_best), Q.n_queries, P, Q, O, t1, err, s);
  else  // long lists: warp-cooperative walk
    e = n_best <= kT1CompactGenomes
            ? launch_smem(k_summin_smem<kT1Threads, kT1MinBlocks, kT1Cap, kT1Out, true, false, false, kT1Used, true>,
                          L, "summin_bh", kT1Threads, T1::bytes(n_best), Q.n_queries, P, Q, O, t1, err, s)
        : n_best <= kT1MidGenomes
            ? launch_smem(k_summin_smem<kT1Threads, kT1MinBlocks, kT1Cap, kT1OutMid, true, false, false, kT1UsedMid, true>,
                          L, "summin_bh", kT1Threads, T1M::bytes(n_best), Q.n_queries, P, Q, O, t1, err, s)
            : launch_smem(
                  k_summin_smem<kT1Threads, kT1MinBlocks, kT1Cap, kT1OutFull, true, false, false, kT1UsedFull, true>, L,
                  "summin_bh", kT1Threads, T1F::bytes(n_best), Q.n_queries, P, Q, O, t1, err, s);
  if (e != cudaSuccess) return e;
  // tier 2: one 1024-thread block per SM over the deferred queries (exits at once if none)
  if (emit_all)
    e = launch_smem(k_summin_smem<kT2Threads, 1, kT2Cap, kT2OutEmit, false, true>, L, "summin_pairs_t2", kT2Threads,
                    T2E::bytes(n_best), Q.n_queries, P, Q, O, t2, err, s);
  else
    e = launch_smem(k_summin_smem<kT2Threads, 1, kT2Cap, kT2Out, false, false>, L, "summin_bh_t2", kT2Threads,
                    T2::bytes(n_best), Q.n_queries, P, Q, O, t2, err, s);
  return e;
}

size_t summin_global_smem_bytes(uint32_t n_genomes) {
  return Chunk<256>::kBytes + (size_t)(n_genomes ? n_genomes : 1) * 12 + 4;
}

cudaError_t run_summin_global(Launcher* L, const ProfilesView& P, const QuerySet& Q, const HitsOut& O,
                              const BigScratch& B, uint32_t n_ctas, DevErr* err, bool emit_all, cudaStream_t s) {
  const size_t smem = summin_global_smem_bytes(Q.all_pairs ? P.n_genomes : 1u);
  TierIO t3{O.def2, O.n_def2, nullptr, nullptr};
  const char* name = Q.filter ? "summin_bh_f_t3" : (emit_all ? "summin_pairs_t3" : "summin_bh_t3");
  cudaError_t e;
  if (Q.filter) {
    if (emit_all || !B.vpa || !B.vpb) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(k_summin_global<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if ((e = launch_begin(L, name)) != cudaSuccess) return e;
    k_summin_global<false, true><<<n_ctas, 256, smem, s>>>(P, Q, O, t3, B, err);
    return launch_end(L, name);
  }
  if (emit_all)
    e = cudaFuncSetAttribute(k_summin_global<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else
    e = cudaFuncSetAttribute(k_summin_global<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if ((e = launch_begin(L, name)) != cudaSuccess) return e;
  if (emit_all)
    k_summin_global<true><<<n_ctas, 256, smem, s>>>(P, Q, O, t3, B, err);
  else
    k_summin_global<false><<<n_ctas, 256, smem, s>>>(P, Q, O, t3, B, err);
  return launch_end(L, name);
}

}  // namespace pdg
