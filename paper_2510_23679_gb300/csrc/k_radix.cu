// k_radix.cu -- stable LSD radix sort of 64-bit records by their high word,
// used to transpose the multiplicity vectors into the inverted index.
//
// The records (k-mer id << 32 | packed posting) arrive in gene order, so a
// stable sort by id leaves every posting list ascending by gene.  Each pass
// sorts by one digit of up to 9 bits:
//   upsweep    per tile of kTile records: digit counts (shared-memory
//              counters), stored digit-major;
//   (scan)     exclusive prefix over (digit, tile): the global start of each
//              tile's run of each digit;
//   downsweep  per tile: stable ranks within each warp from the lanes holding
//              the same digit (one ballot per digit bit), then per-digit
//              offsets across the warps; the tile is
//              staged in shared memory in sorted order and written out, so
//              consecutive threads store consecutive addresses of a digit run.
// After the last pass `post_split` peels the low words into the posting array
// and marks the first position of each id in post_ptr.
#include "pd_internal.cuh"

namespace pdg {
namespace {

constexpr int kRThreads = 256;
constexpr int kRWarps = kRThreads / 32;
constexpr int kRItems = 12;                       // records per lane
constexpr uint32_t kTile = kRThreads * kRItems;   // 3072 records per tile
constexpr int kRDownBlocks = 4;                   // resident downsweep blocks per SM (64 registers)
constexpr int kMaxBins = 512;

__device__ __forceinline__ uint32_t digit_of(unsigned long long r, uint32_t shift, uint32_t bins) {
  return ((uint32_t)(r >> 32) >> shift) & (bins - 1u);
}

__global__ void __launch_bounds__(kRThreads)
    k_radix_upsweep(const unsigned long long* __restrict__ in, uint64_t n, uint32_t shift, uint32_t bins,
                    uint32_t n_tiles, uint32_t* __restrict__ counts) {
  __shared__ uint32_t cnt[kMaxBins];
  for (uint32_t d = threadIdx.x; d < bins; d += kRThreads) cnt[d] = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint64_t t0 = (uint64_t)blockIdx.x * kTile + (uint64_t)warp * (kTile / kRWarps);
  unsigned long long xr[kRItems];
#pragma unroll
  for (int r = 0; r < kRItems; ++r) {
    const uint64_t i = t0 + (uint64_t)r * 32 + lane;
    xr[r] = i < n ? in[i] : ~0ull;
  }
#pragma unroll
  for (int r = 0; r < kRItems; ++r)
    if (t0 + (uint64_t)r * 32 + lane < n) atomicAdd(&cnt[digit_of(xr[r], shift, bins)], 1u);
  __syncthreads();
  for (uint32_t d = threadIdx.x; d < bins; d += kRThreads) counts[(uint64_t)d * n_tiles + blockIdx.x] = cnt[d];
}

__global__ void __launch_bounds__(kRThreads, kRDownBlocks)
    k_radix_downsweep(const unsigned long long* __restrict__ in, unsigned long long* __restrict__ out, uint64_t n,
                      uint32_t shift, uint32_t bins, uint32_t n_tiles, const uint32_t* __restrict__ goff) {
  __shared__ uint32_t wcnt[kRWarps][kMaxBins];  // per-warp counts, then per-warp offsets
  __shared__ uint32_t tbase[kMaxBins + 1];      // tile-local start of each digit
  __shared__ uint32_t warp_tmp[kRWarps + 1];
  extern __shared__ unsigned long long stage[];  // kTile records (dynamic: past the 48 KB static limit)
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  for (uint32_t x = threadIdx.x; x < kRWarps * kMaxBins; x += kRThreads) (&wcnt[0][0])[x] = 0;
  __syncthreads();
  const uint64_t tile0 = (uint64_t)blockIdx.x * kTile;
  const uint64_t t0 = tile0 + (uint64_t)warp * (kTile / kRWarps);
  unsigned long long xr[kRItems];
  uint32_t rk[kRItems];
#pragma unroll
  for (int r = 0; r < kRItems; ++r) {
    const uint64_t i = t0 + (uint64_t)r * 32 + lane;
    xr[r] = i < n ? in[i] : 0ull;
  }
  // stable rank of each record among the warp's records of the same digit
#pragma unroll
  for (int r = 0; r < kRItems; ++r) {
    const bool valid = t0 + (uint64_t)r * 32 + lane < n;
    const uint32_t d = valid ? digit_of(xr[r], shift, bins) : 0xFFFFFFFFu;
    // lanes with the same digit: the AND over the digit's bits of each bit's
    // ballot (or its complement); invalid lanes form a group of their own
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
    if (!valid) peers = ~peers;
    for (uint32_t b = 0; (1u << b) < bins; ++b) {
      const bool bit = (d >> b) & 1u;
      const uint32_t bal = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? bal : ~bal;
    }
    const uint32_t leader = (uint32_t)(__ffs(peers) - 1);
    uint32_t base = 0;
    if (valid && lane == leader) {
      base = wcnt[warp][d];
      wcnt[warp][d] = base + (uint32_t)__popc(peers);
    }
    base = __shfl_sync(0xffffffffu, base, leader);
    rk[r] = base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
  }
  __syncthreads();
  // per digit: exclusive prefix over the warps, and the tile total; thread t
  // owns the consecutive digits 2t and 2t+1 so that a block scan over the
  // threads yields the digits' tile-local starts in digit order
  uint32_t tot[2] = {0u, 0u};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const uint32_t d = 2u * threadIdx.x + (uint32_t)j;
    if (d < bins) {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kRWarps; ++w) {
        const uint32_t c = wcnt[w][d];
        wcnt[w][d] = run;
        run += c;
      }
      tot[j] = run;
    }
  }
  uint32_t all;
  const uint32_t ex = block_exclusive_scan(tot[0] + tot[1], warp_tmp, &all);
  if (2u * threadIdx.x < bins) tbase[2u * threadIdx.x] = ex;
  if (2u * threadIdx.x + 1u < bins) tbase[2u * threadIdx.x + 1u] = ex + tot[0];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRItems; ++r) {
    const bool valid = t0 + (uint64_t)r * 32 + lane < n;
    if (valid) {
      const uint32_t d = digit_of(xr[r], shift, bins);
      stage[tbase[d] + wcnt[warp][d] + rk[r]] = xr[r];
    }
  }
  __syncthreads();
  const uint32_t tile_n = (uint32_t)(n - tile0 < kTile ? n - tile0 : kTile);
  for (uint32_t p = threadIdx.x; p < tile_n; p += kRThreads) {
    const unsigned long long v = stage[p];
    const uint32_t d = digit_of(v, shift, bins);
    out[(uint64_t)goff[(uint64_t)d * n_tiles + blockIdx.x] + (p - tbase[d])] = v;
  }
}

// Sorted records -> postings (low words) and the first position of each id.
// Records with id 0xFFFFFFFF (unused multiplicity-vector slots) sort last;
// the position of the first of them (or n) is the number of postings E.
__global__ void k_post_split(const unsigned long long* __restrict__ rec, uint64_t n, uint64_t n_ids,
                             uint32_t* __restrict__ post, uint32_t* __restrict__ post_ptr) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long v = rec[i];
    const uint32_t id = (uint32_t)(v >> 32);
    const uint32_t prev = i ? (uint32_t)(rec[i - 1] >> 32) : 0xFFFFFFFEu;
    if (id == 0xFFFFFFFFu) {
      if (prev != 0xFFFFFFFFu) post_ptr[n_ids] = (uint32_t)i;
      continue;
    }
    post[i] = (uint32_t)v;
    if (i == 0 || prev != id) post_ptr[id] = (uint32_t)i;
    if (i == n - 1) post_ptr[n_ids] = (uint32_t)n;
  }
}

}  // namespace

size_t radix_counts_words(uint64_t n) {
  const uint64_t n_tiles = (n + kTile - 1) / kTile;
  return (size_t)kMaxBins * (n_tiles ? n_tiles : 1) + 1;
}

cudaError_t run_index_sort(Launcher* L, unsigned long long* a, unsigned long long* b, uint64_t n, uint32_t key_bits,
                           uint32_t* counts, void* scan_tmp, uint64_t n_ids, uint32_t* post, uint32_t* post_ptr,
                           cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint32_t n_tiles = (uint32_t)((n + kTile - 1) / kTile);
  const uint32_t passes = (key_bits + 8) / 9;  // digits of at most 9 bits
  const uint32_t width = passes ? (key_bits + passes - 1) / passes : 1;
  unsigned long long* src = a;
  unsigned long long* dst = b;
  cudaError_t e = cudaFuncSetAttribute(k_radix_downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(kTile * sizeof(unsigned long long)));
  if (e != cudaSuccess) return e;
  for (uint32_t p = 0; p < passes; ++p) {
    const uint32_t shift = p * width;
    const uint32_t w = min(width, key_bits - shift);
    const uint32_t bins = 1u << w;
    if ((e = launch_begin(L, "radix_upsweep")) != cudaSuccess) return e;
    k_radix_upsweep<<<n_tiles, kRThreads, 0, s>>>(src, n, shift, bins, n_tiles, counts);
    if ((e = launch_end(L, "radix_upsweep")) != cudaSuccess) return e;
    if ((e = scan_u32(L, counts, (uint64_t)bins * n_tiles, counts, scan_tmp, s)) != cudaSuccess) return e;
    if ((e = launch_begin(L, "radix_downsweep")) != cudaSuccess) return e;
    k_radix_downsweep<<<n_tiles, kRThreads, kTile * sizeof(unsigned long long), s>>>(src, dst, n, shift, bins,
                                                                                     n_tiles, counts);
    if ((e = launch_end(L, "radix_downsweep")) != cudaSuccess) return e;
    unsigned long long* t = src;
    src = dst;
    dst = t;
  }
  const unsigned grid = (unsigned)((n + 255) / 256 < 152u * 16u ? (n + 255) / 256 : 152u * 16u);
  if ((e = launch_begin(L, "post_split")) != cudaSuccess) return e;
  k_post_split<<<grid, 256, 0, s>>>(src, n, n_ids, post, post_ptr);
  return launch_end(L, "post_split");
}

}  // namespace pdg
