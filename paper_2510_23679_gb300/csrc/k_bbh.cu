// k_bbh.cu -- Bidirectional Best Hits ("Bidirectional Best Hit extraction
// phase", Algorithm 3, Eq. (9)) and compaction of Best Hit rows into CSR.
//
// Best Hit rows are sorted by target gene.  For a hit a -> b the mutual check
// looks a up (binary search) in b's own Best Hit row towards a's genome: the
// pair is a BBH exactly when it is there.  (Algorithm 3 also compares S[l,k]
// with the column maximum; with a symmetric similarity that is the same
// condition as l in A_ji[k], so one test suffices.)  One warp per row:
// count pass (flags + per-row counts), a prefix sum, then a write pass, so
// pairs come out in ascending (a, b) order without a sort.
#include "pd_internal.cuh"

namespace pdg {
namespace {

__device__ __forceinline__ uint32_t row_gene(const BbhRows& R, uint32_t x) {
  if (R.all_pairs) return x;
  return x < R.nA ? R.qa0 + x : R.qb0 + (x - R.nA);
}

// Does row x emit its pairs?  All form: only towards genomes after its own
// (each unordered pair once).  Pair form: only the rows of the first genome.
__device__ __forceinline__ bool row_emits(const BbhRows& R, uint32_t x) { return R.all_pairs || x < R.nA; }

__device__ __forceinline__ uint32_t partner_row(const BbhRows& R, uint32_t b) {
  return R.all_pairs ? b : R.nA + (b - R.qb0);
}

// Is a in the ascending row hit_b[off .. off+n)?  Rows of the all-pairs form
// hold about one target per genome, so gene ids spread evenly over the row:
// an interpolation guess lands next to a, a galloping step brackets it and a
// binary search finishes (two to four reads instead of a full binary search).
__device__ __forceinline__ bool row_contains(const uint32_t* __restrict__ hit_b, unsigned long long off, uint32_t n,
                                             uint32_t a) {
  if (n == 0) return false;
  const uint32_t first = hit_b[off], last = hit_b[off + n - 1];
  if (a < first || a > last) return false;
  if (a == first || a == last) return true;
  // here first < a < last, so n >= 3 and the answer lies in [1, n-1)
  const uint32_t g = (uint32_t)(((unsigned long long)(a - first) * (n - 1)) / (last - first));
  const uint32_t v = hit_b[off + g];
  if (v == a) return true;
  uint32_t lo, hi;  // a, if present, is in [lo, hi)
  if (v < a) {
    lo = g + 1;
    hi = n - 1;
    for (uint32_t step = 1; g + step < n - 1; step <<= 1) {
      const uint32_t w = hit_b[off + g + step];
      if (w == a) return true;
      if (w > a) {
        hi = g + step;
        break;
      }
      lo = g + step + 1;
    }
  } else {
    lo = 1;
    hi = g;
    for (uint32_t step = 1; step < g; step <<= 1) {
      const uint32_t w = hit_b[off + g - step];
      if (w == a) return true;
      if (w < a) {
        lo = g - step + 1;
        break;
      }
      hi = g - step;
    }
  }
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (hit_b[off + mid] < a) lo = mid + 1; else hi = mid;
  }
  return lo < n && hit_b[off + lo] == a;
}

__global__ void __launch_bounds__(256) k_bbh_count(BbhRows R, uint8_t* __restrict__ flags, uint32_t* __restrict__ row_cnt) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < R.n_rows; x += warps) {
    uint32_t cnt = 0;
    if (row_emits(R, x)) {
      const uint32_t a = row_gene(R, x);
      const unsigned long long off = R.row_off[x];
      const uint32_t n = R.row_len[x];
      // all form: a pair is emitted from the row of its gene in the earlier
      // genome; genes are numbered genome by genome, so a target lies in a
      // later genome exactly when it is past the end of a's genome
      const uint32_t own_end = (R.all_pairs && !R.paralog) ? (uint32_t)R.genome_ptr[R.gene_genome[a] + 1] : 0u;
      for (uint32_t e0 = 0; e0 < n; e0 += 32) {
        const uint32_t e = e0 + lane;
        bool f = false;
        if (e < n) {
          const uint32_t b = R.hit_b[off + e];
          if (!R.all_pairs || (R.paralog ? b > a : b >= own_end)) {
            const uint32_t y = partner_row(R, b);
            f = row_contains(R.hit_b, R.row_off[y], R.row_len[y], a);
          }
          flags[off + e] = f ? 1 : 0;
        }
        cnt += __popc(__ballot_sync(0xffffffffu, f));
      }
    }
    if (lane == 0) row_cnt[x] = cnt;
  }
}

__global__ void __launch_bounds__(256) k_bbh_write(BbhRows R, const uint8_t* __restrict__ flags,
                                                   const uint32_t* __restrict__ row_start, uint32_t a_base,
                                                   uint32_t b_base, int32_t* __restrict__ out_a,
                                                   int32_t* __restrict__ out_b) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < R.n_rows; x += warps) {
    if (!row_emits(R, x)) continue;
    const uint32_t a = row_gene(R, x);
    const unsigned long long off = R.row_off[x];
    const uint32_t n = R.row_len[x];
    uint32_t dst = row_start[x];
    for (uint32_t e0 = 0; e0 < n; e0 += 32) {
      const uint32_t e = e0 + lane;
      const bool f = (e < n) && flags[off + e];
      const uint32_t m = __ballot_sync(0xffffffffu, f);
      if (f) {
        const uint32_t at = dst + __popc(m & ((1u << lane) - 1u));
        out_a[at] = (int32_t)(a - a_base);
        out_b[at] = (int32_t)(R.hit_b[off + e] - b_base);
      }
      dst += __popc(m);
    }
  }
}

__global__ void __launch_bounds__(256) k_gather_rows(uint32_t n_rows, const unsigned long long* __restrict__ row_off,
                                                     const uint32_t* __restrict__ row_len,
                                                     const unsigned long long* __restrict__ row_ptr,
                                                     const uint32_t* __restrict__ in_b, const uint32_t* __restrict__ in_s,
                                                     uint32_t col_base, int32_t* __restrict__ out_cols,
                                                     uint32_t* __restrict__ out_s) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n_rows; x += warps) {
    const unsigned long long src = row_off[x], dst = row_ptr[x];
    for (uint32_t e = lane; e < row_len[x]; e += 32) {
      if (out_cols) out_cols[dst + e] = (int32_t)(in_b[src + e] - col_base);
      if (out_s) out_s[dst + e] = in_s[src + e];
    }
  }
}

unsigned warp_grid(uint64_t rows) {
  uint64_t b = (rows * 32 + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152u * 16u) b = 152u * 16u;
  return (unsigned)b;
}

}  // namespace

cudaError_t run_gather_rows(Launcher* L, uint32_t n_rows, const unsigned long long* row_off, const uint32_t* row_len,
                            const unsigned long long* row_ptr, const uint32_t* in_b, const uint32_t* in_s,
                            uint32_t col_base, int32_t* out_cols, uint32_t* out_s, cudaStream_t s) {
  cudaError_t e = launch_begin(L, "gather_rows");
  if (e != cudaSuccess) return e;
  k_gather_rows<<<warp_grid(n_rows), 256, 0, s>>>(n_rows, row_off, row_len, row_ptr, in_b, in_s, col_base, out_cols,
                                                  out_s);
  return launch_end(L, "gather_rows");
}

cudaError_t run_bbh_count(Launcher* L, const BbhRows& R, uint8_t* flags_by_hit, uint32_t* row_cnt, cudaStream_t s) {
  cudaError_t e = launch_begin(L, "bbh_count");
  if (e != cudaSuccess) return e;
  k_bbh_count<<<warp_grid(R.n_rows), 256, 0, s>>>(R, flags_by_hit, row_cnt);
  return launch_end(L, "bbh_count");
}

cudaError_t run_bbh_write(Launcher* L, const BbhRows& R, const uint8_t* flags_by_hit, const uint32_t* row_start,
                          uint32_t a_base, uint32_t b_base, int32_t* out_a, int32_t* out_b, cudaStream_t s) {
  cudaError_t e = launch_begin(L, "bbh_write");
  if (e != cudaSuccess) return e;
  k_bbh_write<<<warp_grid(R.n_rows), 256, 0, s>>>(R, flags_by_hit, row_start, a_base, b_base, out_a, out_b);
  return launch_end(L, "bbh_write");
}

}  // namespace pdg
