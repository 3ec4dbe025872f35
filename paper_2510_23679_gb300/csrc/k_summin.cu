// k_summin.cu -- sum-min by inverted-index scatter, fused with Best Hit
// selection ("Best Hit detection phase", Algorithm 2, Eqs. (5) and (8)).
//
// One thread block owns one query gene a at a time:
//   1. stage a chunk of a's multiplicity vector (id, mult_a) in shared memory
//      with the posting range of each id (restricted by binary search to the
//      target gene range in the pair form) and a block prefix sum of the
//      range lengths, so that the chunk's postings form one flat index space;
//   2. every thread walks flat posting indices (consecutive threads read
//      consecutive postings: coalesced), unpacks (b, mult_b) and adds
//      min(mult_a, mult_b) to b's accumulator in a shared-memory open-
//      addressing hash table: after all chunks, acc[b] = s(a, b) =
//      sum over shared k-mers of min(mult) (Eq. (5) numerator), exactly;
//   3. Best Hits: per target genome, the maximum of s / (La + Lb - s) is kept
//      as a (s, den) pair updated by compare-and-swap with a 64-bit
//      cross-multiplication order; every accumulator whose ratio equals its
//      genome's maximum (again by cross-multiplication) is a Best Hit (Eq. (8),
//      ties kept); the block sorts them by gene and appends them to the output.
// The similarity matrix S_ij is never materialised: only pairs sharing a
// k-mer are touched.  A query whose accumulator would pass 3/4 of the shared
// table, or whose Best Hit list does not fit, is deferred to the second tier,
// which runs the same code with the table in global memory sized for every
// possible target, so results are exact for any input.
#include <algorithm>

#include "pd_internal.cuh"

namespace pdg {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kCap = 4096;     // shared hash slots (power of two)
constexpr uint32_t kChunk = 1024;   // query k-mers staged per round
constexpr uint32_t kItems = kChunk / kThreads;
constexpr uint32_t kOutCap = 1024;  // Best Hit entries per query in the shared tier
constexpr uint32_t kMinCap = 64;

struct Scalars {
  uint32_t n_used;
  uint32_t n_out;
  uint32_t overflow;
  uint32_t base_lo, base_hi;
  uint32_t warp_tmp[kThreads / 32 + 1];
};

__device__ __forceinline__ uint32_t hash_gene(uint32_t b) {
  uint32_t h = b * 0x9E3779B1u;
  return h ^ (h >> 15);
}

// Add m to the accumulator of gene b.  Returns false when the table is over
// its load limit or full (the caller defers the query).
__device__ __forceinline__ bool acc_add(uint32_t* keys, uint32_t* vals, uint32_t mask, uint32_t b, uint32_t m,
                                        uint32_t* n_used, uint32_t limit) {
  uint32_t h = hash_gene(b) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    uint32_t k = *((volatile uint32_t*)&keys[h]);
    if (k == b) {
      atomicAdd(&vals[h], m);
      return true;
    }
    if (k == kEmpty) {
      uint32_t prev = atomicCAS(&keys[h], kEmpty, b);
      if (prev == kEmpty) {
        atomicAdd(&vals[h], m);
        return atomicAdd(n_used, 1u) < limit;
      }
      if (prev == b) {
        atomicAdd(&vals[h], m);
        return true;
      }
    }
    h = (h + 1) & mask;
  }
  return false;
}

__device__ __forceinline__ uint32_t lower_bound_post(const uint32_t* __restrict__ post, uint32_t lo, uint32_t hi,
                                                     unsigned long long key) {
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if ((unsigned long long)post[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t mv_count_of(const ProfilesView& P, uint32_t g, uint32_t id) {
  uint32_t lo = P.win_off[g], end = lo + P.mv_len[g], hi = end;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (P.mv_id[mid] < id) lo = mid + 1; else hi = mid;
  }
  return (lo < end && P.mv_id[lo] == id) ? P.mv_cnt[lo] : 0u;
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

template <bool kBig, bool kEmitAll>
__device__ __forceinline__ void process_query(uint32_t qi, const ProfilesView& P, const QuerySet& Q,
                                              const HitsOut& O, DevErr* err, uint32_t* keys, uint32_t* vals,
                                              uint32_t cap_max, unsigned long long* out, uint32_t out_cap,
                                              uint32_t* c_lo, uint32_t* c_off, uint16_t* c_cnt,
                                              unsigned long long* best, Scalars* sh) {
  // ---- query gene and its targets
  uint32_t a, tlo, thi, own0 = 0, own1 = 0;
  if (Q.all_pairs) {
    a = Q.q0 + qi;
    const uint32_t gg = P.gene_genome[a];
    own0 = (uint32_t)P.genome_ptr[gg];
    own1 = (uint32_t)P.genome_ptr[gg + 1];
    tlo = 0;
    thi = P.n_genes;
  } else if (qi < Q.nA) {
    a = Q.qa0 + qi;
    tlo = Q.ta0;
    thi = Q.ta1;
  } else {
    a = Q.qb0 + (qi - Q.nA);
    tlo = Q.tb0;
    thi = Q.tb1;
  }
  const uint32_t m0 = P.win_off[a], E = P.mv_len[a], La_a = P.La[a];
  const uint32_t cnt_mask = (1u << P.cnt_bits) - 1u;
  const unsigned long long key_lo = (unsigned long long)tlo << P.cnt_bits;
  const unsigned long long key_hi = (unsigned long long)thi << P.cnt_bits;
  const uint32_t tid = threadIdx.x;

  if (tid == 0) {
    sh->n_used = 0;
    sh->n_out = 0;
    sh->overflow = 0;
  }
  __syncthreads();
  uint32_t cap = cap_max;
  unsigned long long walked = 0;
  for (uint32_t c0 = 0; c0 < E; c0 += kChunk) {
    const uint32_t n_c = min(kChunk, E - c0);
    // ---- stage the chunk: posting ranges and their prefix sum
    uint32_t len_loc[kItems];
    uint32_t my_sum = 0;
#pragma unroll
    for (uint32_t r = 0; r < kItems; ++r) {
      const uint32_t e = tid * kItems + r;
      uint32_t len = 0;
      if (e < n_c) {
        const uint32_t id = P.mv_id[m0 + c0 + e];
        uint32_t lo = P.post_ptr[id], hi = P.post_ptr[id + 1];
        if (!Q.all_pairs) {
          lo = lower_bound_post(P.post, lo, hi, key_lo);
          hi = lower_bound_post(P.post, lo, hi, key_hi);
        }
        c_lo[e] = lo;
        c_cnt[e] = P.mv_cnt[m0 + c0 + e];
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
      if (e < n_c) c_off[e] = run;
      run += len_loc[r];
    }
    if (tid == 0) c_off[n_c] = J_c;
    // ---- size and clear the accumulator before the first chunk
    if (c0 == 0) {
      if (E <= kChunk && J_c < (cap_max >> 1)) cap = max(kMinCap, next_pow2(2u * J_c));
      for (uint32_t h = tid; h < cap; h += kThreads) {
        keys[h] = kEmpty;
        vals[h] = 0;
      }
    }
    __syncthreads();
    walked += J_c;
    const uint32_t mask = cap - 1u;
    const uint32_t limit = (cap >> 2) * 3u;
    // ---- walk the chunk's postings
    for (uint32_t t = tid; t < J_c; t += kThreads) {
      uint32_t lo = 0, hi = n_c;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (c_off[mid] <= t) lo = mid; else hi = mid;
      }
      const uint32_t p = P.post[c_lo[lo] + (t - c_off[lo])];
      const uint32_t b = p >> P.cnt_bits;
      if (Q.all_pairs && b >= own0 && b < own1) continue;
      const uint32_t ca = c_cnt[lo];
      uint32_t cb = p & cnt_mask;
      if (cb == P.cnt_cap && ca > cb) cb = mv_count_of(P, b, P.mv_id[m0 + c0 + lo]);
      if (!acc_add(keys, vals, mask, b, min(ca, cb), &sh->n_used, limit)) sh->overflow = 1;
    }
    __syncthreads();
    if (sh->overflow) break;
  }

  bool defer = sh->overflow != 0;
  uint32_t n_out = 0;
  if (!defer && E > 0) {
    if (kEmitAll) {
      // every accumulator is an output (the sum-min test hook)
      for (uint32_t h = tid; h < cap; h += kThreads) {
        const uint32_t b = keys[h];
        if (b == kEmpty) continue;
        const uint32_t slot = atomicAdd(&sh->n_out, 1u);
        if (slot < out_cap) out[slot] = ((unsigned long long)b << 32) | vals[h];
      }
    } else {
      // ---- per target genome: the maximum ratio, then every entry at it
      const uint32_t n_best = Q.all_pairs ? P.n_genomes : 1u;
      for (uint32_t j = tid; j < n_best; j += kThreads) best[j] = 0ull;
      __syncthreads();
      for (uint32_t h = tid; h < cap; h += kThreads) {
        const uint32_t b = keys[h];
        if (b == kEmpty) continue;
        const uint32_t s = vals[h];
        const uint32_t den = La_a + P.La[b] - s;
        best_update(&best[Q.all_pairs ? (uint32_t)P.gene_genome[b] : 0u], s, den);
      }
      __syncthreads();
      for (uint32_t h = tid; h < cap; h += kThreads) {
        const uint32_t b = keys[h];
        if (b == kEmpty) continue;
        const uint32_t s = vals[h];
        const uint32_t den = La_a + P.La[b] - s;
        const unsigned long long bv = best[Q.all_pairs ? (uint32_t)P.gene_genome[b] : 0u];
        if (ratio_equal(s, den, (uint32_t)(bv >> 32), (uint32_t)bv)) {
          const uint32_t slot = atomicAdd(&sh->n_out, 1u);
          if (slot < out_cap) out[slot] = ((unsigned long long)b << 32) | s;
        }
      }
    }
    __syncthreads();
    n_out = sh->n_out;
    if (n_out > out_cap) defer = true;
  }

  if (defer) {
    if (kBig) {  // cannot happen: the large tier is sized for every target
      if (tid == 0) raise_error(err, PD_ERR_INTERNAL, qi);
    } else if (tid == 0) {
      O.deferred[atomicAdd(O.n_deferred, 1u)] = qi;
    }
    if (tid == 0) {
      O.row_off[qi] = 0;
      O.row_len[qi] = 0;
    }
    __syncthreads();
    return;
  }

  // ---- sort the hits by gene and append them
  if (n_out > 1) {
    const uint32_t n2 = next_pow2(n_out);
    for (uint32_t x = n_out + tid; x < n2; x += kThreads) out[x] = ~0ull;
    __syncthreads();
    block_bitonic_sort(out, n2);
  }
  if (tid == 0) {
    const unsigned long long base = atomicAdd(O.cursor, (unsigned long long)n_out);
    sh->base_lo = (uint32_t)base;
    sh->base_hi = (uint32_t)(base >> 32);
    O.row_off[qi] = base;
    O.row_len[qi] = n_out;
    atomicAdd(O.walked, walked);
  }
  __syncthreads();
  const unsigned long long base = ((unsigned long long)sh->base_hi << 32) | sh->base_lo;
  if (base + n_out <= O.out_cap) {
    for (uint32_t x = tid; x < n_out; x += kThreads) {
      O.out_b[base + x] = (uint32_t)(out[x] >> 32);
      O.out_s[base + x] = (uint32_t)out[x];
    }
  }
  __syncthreads();
}

template <bool kEmitAll>
__host__ __device__ constexpr uint32_t out_cap_smem() {
  return kEmitAll ? kCap : kOutCap;
}

template <bool kEmitAll>
__host__ __device__ constexpr size_t union_bytes() {
  constexpr size_t chunk = (size_t)kChunk * 4 + (size_t)(kChunk + 1) * 4 + (size_t)kChunk * 2;
  constexpr size_t outb = (size_t)out_cap_smem<kEmitAll>() * 8;
  return ((chunk > outb ? chunk : outb) + 15) & ~(size_t)15;
}

template <bool kEmitAll>
__global__ void __launch_bounds__(kThreads) k_summin_bh(ProfilesView P, QuerySet Q, HitsOut O, DevErr* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Scalars sh;
  uint32_t* keys = (uint32_t*)smem;
  uint32_t* vals = keys + kCap;
  unsigned char* uni = (unsigned char*)(vals + kCap);
  unsigned long long* out = (unsigned long long*)uni;
  uint32_t* c_lo = (uint32_t*)uni;
  uint32_t* c_off = c_lo + kChunk;
  uint16_t* c_cnt = (uint16_t*)(c_off + kChunk + 1);
  unsigned long long* best = (unsigned long long*)(uni + union_bytes<kEmitAll>());
  for (uint32_t qi = blockIdx.x; qi < Q.n_queries; qi += gridDim.x)
    process_query<false, kEmitAll>(qi, P, Q, O, err, keys, vals, kCap, out, out_cap_smem<kEmitAll>(), c_lo, c_off,
                                   c_cnt, best, &sh);
}

template <bool kEmitAll>
__global__ void __launch_bounds__(kThreads) k_summin_bh_big(ProfilesView P, QuerySet Q, HitsOut O, BigScratch B,
                                                            DevErr* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Scalars sh;
  uint32_t* c_lo = (uint32_t*)smem;
  uint32_t* c_off = c_lo + kChunk;
  uint16_t* c_cnt = (uint16_t*)(c_off + kChunk + 1);
  unsigned long long* best = (unsigned long long*)(smem + union_bytes<false>());
  uint32_t* keys = B.keys + (size_t)blockIdx.x * B.cap;
  uint32_t* vals = B.vals + (size_t)blockIdx.x * B.cap;
  unsigned long long* out = B.out + (size_t)blockIdx.x * B.out_cap;
  const uint32_t n_def = *O.n_deferred;
  for (uint32_t x = blockIdx.x; x < n_def; x += gridDim.x)
    process_query<true, kEmitAll>(O.deferred[x], P, Q, O, err, keys, vals, B.cap, out, B.out_cap, c_lo, c_off, c_cnt,
                                  best, &sh);
}

}  // namespace

size_t summin_smem_bytes(uint32_t n_genomes, bool emit_all) {
  const size_t best = (size_t)(n_genomes ? n_genomes : 1) * 8;
  return (size_t)kCap * 8 + (emit_all ? union_bytes<true>() : union_bytes<false>()) + best;
}

cudaError_t run_summin_bh(Launcher* L, const ProfilesView& P, const QuerySet& Q, const HitsOut& O, DevErr* err,
                          bool emit_all, cudaStream_t s) {
  if (Q.n_queries == 0) return cudaSuccess;
  const size_t smem = summin_smem_bytes(P.n_genomes, emit_all);
  const char* name = emit_all ? "summin_pairs" : "summin_bh";
  cudaError_t e;
  if (emit_all)
    e = cudaFuncSetAttribute(k_summin_bh<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else
    e = cudaFuncSetAttribute(k_summin_bh<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if (emit_all)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_summin_bh<true>, kThreads, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_summin_bh<false>, kThreads, smem);
  int dev = 0, n_sm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::min<uint64_t>(Q.n_queries, (uint64_t)n_sm * (per_sm > 0 ? per_sm : 1) * 8);
  if ((e = launch_begin(L, name)) != cudaSuccess) return e;
  if (emit_all)
    k_summin_bh<true><<<grid, kThreads, smem, s>>>(P, Q, O, err);
  else
    k_summin_bh<false><<<grid, kThreads, smem, s>>>(P, Q, O, err);
  return launch_end(L, name);
}

cudaError_t run_summin_bh_big(Launcher* L, const ProfilesView& P, const QuerySet& Q, const HitsOut& O,
                              const BigScratch& B, uint32_t n_ctas, DevErr* err, bool emit_all, cudaStream_t s) {
  const size_t smem = union_bytes<false>() + (size_t)(P.n_genomes ? P.n_genomes : 1) * 8;
  const char* name = emit_all ? "summin_pairs_big" : "summin_bh_big";
  cudaError_t e;
  if (emit_all)
    e = cudaFuncSetAttribute(k_summin_bh_big<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else
    e = cudaFuncSetAttribute(k_summin_bh_big<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if ((e = launch_begin(L, name)) != cudaSuccess) return e;
  if (emit_all)
    k_summin_bh_big<true><<<n_ctas, kThreads, smem, s>>>(P, Q, O, B, err);
  else
    k_summin_bh_big<false><<<n_ctas, kThreads, smem, s>>>(P, Q, O, B, err);
  return launch_end(L, name);
}

}  // namespace pdg
