// k_sym.cu -- Best Hit rows of the symmetric all-pairs form.
//
// The similarity J is symmetric (Eq. (5)), so S_ji is the transpose of S_ij
// and the all-against-all comparison needs each unordered genome pair walked
// once.  In the symmetric form (QuerySet::symbest) query a of genome i walks
// only the targets in genomes j > i and emits its forward Best Hits there
// (Eq. (8)); while it does so, every candidate b in such a genome j keeps the
// best ratio it reaches over the genes of G_i, with the gene that reaches it,
// and a list of exact ties.  That maximum over a column of S_ij gives the Best
// Hits of b in G_i (the reverse direction: Algorithm 3's column maximum).
//
// Row b of the result is then its Best Hits in the genomes before its own
// (the stored maxima and the ties that equal them, ascending) followed by its
// forward Best Hits in the genomes after its own -- ascending overall, since
// genes are numbered genome by genome.
#include "pd_internal.cuh"

namespace pdg {
namespace {

__device__ __forceinline__ void unpack(unsigned long long w, uint32_t* s, uint32_t* den, uint32_t* a) {
  *s = (uint32_t)(w >> 48);
  *den = (uint32_t)(w >> 31) & 0x1FFFFu;
  *a = (uint32_t)w & 0x7FFFFFFFu;
}

// One thread per gene: stored maxima of the genomes before its own (the
// maxima are genome-major, so neighbouring threads read neighbouring words).
__global__ void __launch_bounds__(256) k_sym_count(SymRows R, uint32_t* __restrict__ stored) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < R.n_genes; b += gridDim.x * blockDim.x) {
    const uint32_t gb = R.gene_genome[b];
    uint32_t n = 0;
    for (uint32_t g = 0; g < gb; ++g) n += R.symbest[(size_t)g * R.n_genes + b] != 0ull ? 1u : 0u;
    stored[b] = n;
  }
}

// Is (b, a) new to the set?  Open addressing over `keys` (a power of two at
// least twice the ties, all-ones = empty), so a probe always ends.
__device__ __forceinline__ bool first_insert(unsigned long long* keys, unsigned long long mask,
                                             unsigned long long key) {
  unsigned long long h = (key * 0x9E3779B97F4A7C15ull) & mask;
  for (unsigned long long probe = 0; probe <= mask; ++probe) {
    const unsigned long long prev = atomicCAS(&keys[h], ~0ull, key);
    if (prev == ~0ull) return true;
    if (prev == key) return false;
    h = (h + 1) & mask;
  }
  return false;
}

// One thread per tie (b << 32 | a, s): valid when its ratio equals the final
// stored maximum of (b, genome of a), it is not the stored pair itself, and
// it is the first record of the pair (a query that a tier hands to the next
// after its Best Hit passes records its ties again).
__global__ void k_sym_ties(SymRows R, uint32_t* __restrict__ tiecnt, uint8_t* __restrict__ tie_ok) {
  for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < R.n_ties;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long r = R.tie_rec[2 * t];
    const uint32_t b = (uint32_t)(r >> 32), a = (uint32_t)r, s = (uint32_t)R.tie_rec[2 * t + 1];
    const unsigned long long w = R.symbest[(size_t)R.gene_genome[a] * R.n_genes + b];
    uint32_t ms, md, ma;
    unpack(w, &ms, &md, &ma);
    const bool ok = w != 0ull && ma != a && ratio_equal(s, R.La[a] + R.La[b] - s, ms, md) &&
                    first_insert(R.tie_set, R.tie_set_mask, r);
    tie_ok[t] = ok ? 1 : 0;
    if (ok) atomicAdd(&tiecnt[b], 1u);
  }
}

__global__ void k_sym_total(SymRows R, const uint32_t* __restrict__ stored, const uint32_t* __restrict__ tiecnt,
                            uint32_t* __restrict__ total) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < R.n_genes; b += gridDim.x * blockDim.x)
    total[b] = stored[b] + tiecnt[b] + R.fwd_len[b];
}

// One thread per gene: the stored maxima in genome order.
__global__ void __launch_bounds__(256)
    k_sym_write_rev(SymRows R, const unsigned long long* __restrict__ row_ptr, uint32_t* __restrict__ out_b,
                    uint32_t* __restrict__ out_s) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < R.n_genes; b += gridDim.x * blockDim.x) {
    const uint32_t gb = R.gene_genome[b];
    unsigned long long at = row_ptr[b];
    for (uint32_t g = 0; g < gb; ++g) {
      const unsigned long long w = R.symbest[(size_t)g * R.n_genes + b];
      if (w == 0ull) continue;
      uint32_t s, den, a;
      unpack(w, &s, &den, &a);
      out_b[at] = a;
      out_s[at] = s;
      ++at;
    }
  }
}

// The same through shared memory, for datasets of at most kRevTileGenomes
// genomes: a block reads the maxima of 32 consecutive genes genome by genome
// (coalesced) into a tile, then one warp per gene writes its row part
// (coalesced).  Genes are numbered genome by genome, so the tile's last gene
// has the largest genome of the 32.
constexpr uint32_t kRevTileGenomes = 372;  // 372 x 33 x 8 bytes < 96 KB of shared memory
__global__ void __launch_bounds__(256)
    k_sym_write_rev_tile(SymRows R, const unsigned long long* __restrict__ row_ptr, uint32_t* __restrict__ out_b,
                         uint32_t* __restrict__ out_s) {
  extern __shared__ unsigned long long tile[];  // [genome][33]
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
  for (uint32_t b0 = blockIdx.x * 32u; b0 < R.n_genes; b0 += gridDim.x * 32u) {
    const uint32_t nb = min(32u, R.n_genes - b0);
    const uint32_t gmax = R.gene_genome[b0 + nb - 1];
    for (uint32_t g = warp; g < gmax; g += n_warps)
      tile[g * 33u + lane] = lane < nb ? R.symbest[(size_t)g * R.n_genes + b0 + lane] : 0ull;
    __syncthreads();
    for (uint32_t j = warp; j < nb; j += n_warps) {
      const uint32_t b = b0 + j, gb = R.gene_genome[b];
      unsigned long long at = row_ptr[b];
      for (uint32_t g0 = 0; g0 < gb; g0 += 32) {
        const uint32_t g = g0 + lane;
        const unsigned long long w = g < gb ? tile[g * 33u + j] : 0ull;
        const uint32_t m = __ballot_sync(0xffffffffu, w != 0ull);
        if (w != 0ull) {
          uint32_t s, den, a;
          unpack(w, &s, &den, &a);
          const unsigned long long x = at + __popc(m & ((1u << lane) - 1u));
          out_b[x] = a;
          out_s[x] = s;
        }
        at += __popc(m);
      }
    }
    __syncthreads();
  }
}

// One warp per gene: the forward part, after the stored maxima and room for
// the gene's ties.
__global__ void __launch_bounds__(256)
    k_sym_write(SymRows R, const uint32_t* __restrict__ stored, const uint32_t* __restrict__ tiecnt,
                const unsigned long long* __restrict__ row_ptr, uint32_t* __restrict__ out_b,
                uint32_t* __restrict__ out_s) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < R.n_genes; b += warps) {
    const unsigned long long base = row_ptr[b];
    const unsigned long long fwd = base + stored[b] + tiecnt[b];
    const unsigned long long fo = R.fwd_off[b];
    const uint32_t fl = R.fwd_len[b];
    for (uint32_t e = lane; e < fl; e += 32) {
      out_b[fwd + e] = R.fwd_b[fo + e];
      out_s[fwd + e] = R.fwd_s[fo + e];
    }
  }
}

// Valid ties go after their gene's stored maxima.
__global__ void k_sym_put_ties(SymRows R, const uint8_t* __restrict__ tie_ok, const uint32_t* __restrict__ stored,
                               const unsigned long long* __restrict__ row_ptr, uint32_t* __restrict__ tie_fill,
                               uint32_t* __restrict__ out_b, uint32_t* __restrict__ out_s) {
  for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < R.n_ties;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    if (!tie_ok[t]) continue;
    const unsigned long long r = R.tie_rec[2 * t];
    const uint32_t b = (uint32_t)(r >> 32), a = (uint32_t)r;
    const unsigned long long at = row_ptr[b] + stored[b] + atomicAdd(&tie_fill[b], 1u);
    out_b[at] = a;
    out_s[at] = (uint32_t)R.tie_rec[2 * t + 1];
  }
}

// One thread per gene with ties: insertion sort of its reverse part by gene
// id (ties are exact equalities of two ratios, so such parts are rare).
__global__ void k_sym_sort_ties(uint32_t n_genes, const uint32_t* __restrict__ stored,
                                const uint32_t* __restrict__ tiecnt, const unsigned long long* __restrict__ row_ptr,
                                uint32_t* __restrict__ out_b, uint32_t* __restrict__ out_s) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n_genes; b += gridDim.x * blockDim.x) {
    if (tiecnt[b] == 0) continue;
    const uint32_t n = stored[b] + tiecnt[b];
    uint32_t* kb = out_b + row_ptr[b];
    uint32_t* ks = out_s + row_ptr[b];
    for (uint32_t i = 1; i < n; ++i) {
      const uint32_t x = kb[i], y = ks[i];
      uint32_t j = i;
      while (j > 0 && kb[j - 1] > x) {
        kb[j] = kb[j - 1];
        ks[j] = ks[j - 1];
        --j;
      }
      kb[j] = x;
      ks[j] = y;
    }
  }
}

// Bidirectional Best Hits of the symmetric form, one warp per forward row:
// a forward Best Hit a -> b (b in a later genome) is a BBH exactly when its
// ratio equals b's maximum over a's genome (Eq. (9): a is then among the Best
// Hits of b in G_i, ties included).  Pass 1 flags and counts, pass 2 writes
// at the row's scanned start, so pairs come out ascending.
__global__ void __launch_bounds__(256) k_sym_bbh_count(SymRows R, uint8_t* __restrict__ flag,
                                                       uint32_t* __restrict__ cnt) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < R.n_genes; a += warps) {
    const uint32_t ga = R.gene_genome[a], La = R.La[a];
    const unsigned long long fo = R.fwd_off[a];
    const uint32_t fl = R.fwd_len[a];
    uint32_t n = 0;
    for (uint32_t e = lane; e < fl; e += 32) {
      const uint32_t b = R.fwd_b[fo + e], sv = R.fwd_s[fo + e];
      const unsigned long long w = R.symbest[(size_t)ga * R.n_genes + b];
      const bool f = ratio_equal(sv, La + R.La[b] - sv, (uint32_t)(w >> 48), (uint32_t)(w >> 31) & 0x1FFFFu);
      flag[fo + e] = f ? 1 : 0;
      n += f ? 1u : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (lane == 0) cnt[a] = n;
  }
}

__global__ void __launch_bounds__(256) k_sym_bbh_write(SymRows R, const uint8_t* __restrict__ flag,
                                                       const uint32_t* __restrict__ start, int32_t* __restrict__ pa,
                                                       int32_t* __restrict__ pb) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < R.n_genes; a += warps) {
    const unsigned long long fo = R.fwd_off[a];
    const uint32_t fl = R.fwd_len[a];
    uint32_t pos = start[a];
    for (uint32_t e0 = 0; e0 < fl; e0 += 32) {
      const uint32_t e = e0 + lane;
      const bool f = e < fl && flag[fo + e];
      const uint32_t m = __ballot_sync(0xffffffffu, f);
      if (f) {
        const uint32_t at = pos + __popc(m & ((1u << lane) - 1u));
        pa[at] = (int32_t)a;
        pb[at] = (int32_t)R.fwd_b[fo + e];
      }
      pos += __popc(m);
    }
  }
}

unsigned grid_of(uint64_t items, unsigned per_block, unsigned cap) {
  uint64_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

}  // namespace

cudaError_t run_sym_count(Launcher* L, const SymRows& R, uint32_t* stored, uint32_t* tiecnt, uint8_t* tie_ok,
                          uint32_t* total, cudaStream_t s) {
  cudaError_t e = launch_begin(L, "sym_count");
  if (e != cudaSuccess) return e;
  k_sym_count<<<grid_of((uint64_t)R.n_genes, 256, 152u * 16u), 256, 0, s>>>(R, stored);
  if ((e = launch_end(L, "sym_count")) != cudaSuccess) return e;
  if (R.n_ties) {
    if ((e = launch_begin(L, "sym_ties")) != cudaSuccess) return e;
    k_sym_ties<<<grid_of(R.n_ties, 256, 152u * 16u), 256, 0, s>>>(R, tiecnt, tie_ok);
    if ((e = launch_end(L, "sym_ties")) != cudaSuccess) return e;
  }
  if ((e = launch_begin(L, "sym_total")) != cudaSuccess) return e;
  k_sym_total<<<grid_of(R.n_genes, 256, 152u * 16u), 256, 0, s>>>(R, stored, tiecnt, total);
  return launch_end(L, "sym_total");
}

cudaError_t run_sym_write(Launcher* L, const SymRows& R, const uint32_t* stored, const uint32_t* tiecnt,
                          const uint8_t* tie_ok, const unsigned long long* row_ptr, uint32_t* tie_fill,
                          uint32_t* out_b, uint32_t* out_s, cudaStream_t s) {
  cudaError_t e = launch_begin(L, "sym_write_rev");
  if (e != cudaSuccess) return e;
  if (R.n_genomes <= kRevTileGenomes) {
    const size_t smem = (size_t)R.n_genomes * 33u * sizeof(unsigned long long);
    if ((e = cudaFuncSetAttribute(k_sym_write_rev_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return e;
    k_sym_write_rev_tile<<<grid_of((uint64_t)R.n_genes, 32, 152u * 8u), 256, smem, s>>>(R, row_ptr, out_b, out_s);
  } else {
    k_sym_write_rev<<<grid_of((uint64_t)R.n_genes, 256, 152u * 16u), 256, 0, s>>>(R, row_ptr, out_b, out_s);
  }
  if ((e = launch_end(L, "sym_write_rev")) != cudaSuccess) return e;
  if ((e = launch_begin(L, "sym_write")) != cudaSuccess) return e;
  k_sym_write<<<grid_of((uint64_t)R.n_genes * 32, 256, 152u * 16u), 256, 0, s>>>(R, stored, tiecnt, row_ptr, out_b,
                                                                                 out_s);
  if ((e = launch_end(L, "sym_write")) != cudaSuccess) return e;
  if (R.n_ties == 0) return cudaSuccess;
  if ((e = launch_begin(L, "sym_put_ties")) != cudaSuccess) return e;
  k_sym_put_ties<<<grid_of(R.n_ties, 256, 152u * 16u), 256, 0, s>>>(R, tie_ok, stored, row_ptr, tie_fill, out_b,
                                                                      out_s);
  if ((e = launch_end(L, "sym_put_ties")) != cudaSuccess) return e;
  if ((e = launch_begin(L, "sym_sort_ties")) != cudaSuccess) return e;
  k_sym_sort_ties<<<grid_of(R.n_genes, 256, 152u * 16u), 256, 0, s>>>(R.n_genes, stored, tiecnt, row_ptr, out_b,
                                                                        out_s);
  return launch_end(L, "sym_sort_ties");
}

cudaError_t run_sym_bbh_count(Launcher* L, const SymRows& R, uint8_t* flag, uint32_t* cnt, uint32_t* start,
                              void* scan_tmp, cudaStream_t s) {
  cudaError_t e = launch_begin(L, "sym_bbh_count");
  if (e != cudaSuccess) return e;
  k_sym_bbh_count<<<grid_of((uint64_t)R.n_genes * 32, 256, 152u * 16u), 256, 0, s>>>(R, flag, cnt);
  if ((e = launch_end(L, "sym_bbh_count")) != cudaSuccess) return e;
  return scan_u32(L, cnt, R.n_genes, start, scan_tmp, s);
}

cudaError_t run_sym_bbh_write(Launcher* L, const SymRows& R, const uint8_t* flag, const uint32_t* start, int32_t* pa,
                              int32_t* pb, cudaStream_t s) {
  cudaError_t e = launch_begin(L, "sym_bbh_write");
  if (e != cudaSuccess) return e;
  k_sym_bbh_write<<<grid_of((uint64_t)R.n_genes * 32, 256, 152u * 16u), 256, 0, s>>>(R, flag, start, pa, pb);
  return launch_end(L, "sym_bbh_write");
}

}  // namespace pdg
