// k_scan.cu -- device-wide exclusive prefix sums (reduce, spine, down-sweep).
//
// Used for: rank bases of the k-mer dictionary blocks (dense ids), posting-list offsets
// from per-id counts, and Best Hit / BBH row offsets.  Three launches: each
// tile of kTile elements is reduced, the tile sums are scanned by one block,
// and each tile is rescanned with its offset.  Loads are striped over the
// block (coalesced); partial sums are 64-bit.
#include "pd_internal.cuh"

namespace pdg {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr uint64_t kTile = (uint64_t)kThreads * kItems;

__device__ __forceinline__ unsigned long long warp_incl_u64(unsigned long long v) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= (uint32_t)o) v += y;
  }
  return v;
}

// Exclusive scan over the block; returns the prefix and writes the total.
__device__ __forceinline__ unsigned long long block_excl_u64(unsigned long long v, unsigned long long* tmp,
                                                             unsigned long long* total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  constexpr uint32_t n_warps = kThreads / 32;
  unsigned long long inc = warp_incl_u64(v);
  if (lane == 31) tmp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = (lane < n_warps) ? tmp[lane] : 0ull;
    unsigned long long wi = warp_incl_u64(w);
    if (lane < n_warps) tmp[lane] = wi - w;
    if (lane == n_warps - 1) tmp[n_warps] = wi;
  }
  __syncthreads();
  unsigned long long r = tmp[warp] + inc - v;
  *total = tmp[n_warps];
  __syncthreads();
  return r;
}

// Set bits of dictionary block i (its words 1..7; word 0 receives the scan).
struct DictIn {
  const uint32_t* d;
  __device__ __forceinline__ unsigned long long operator()(uint64_t i) const {
    const uint32_t* b = d + i * 8;
    uint32_t n = 0;
#pragma unroll
    for (int w = 1; w < 8; ++w) n += (uint32_t)__popc(b[w]);
    return n;
  }
};
struct U32In {
  const uint32_t* a;
  __device__ __forceinline__ unsigned long long operator()(uint64_t i) const { return a[i]; }
};

template <typename In>
__global__ void __launch_bounds__(kThreads) k_scan_reduce(In in, uint64_t n, unsigned long long* partial) {
  __shared__ unsigned long long tmp[kThreads / 32 + 1];
  const uint64_t base = (uint64_t)blockIdx.x * kTile;
  unsigned long long sum = 0;
#pragma unroll 4
  for (int r = 0; r < kItems; ++r) {
    uint64_t i = base + (uint64_t)r * kThreads + threadIdx.x;
    if (i < n) sum += in(i);
  }
  unsigned long long total;
  block_excl_u64(sum, tmp, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// One block scans the tile sums in place (exclusive) and stores the total.
__global__ void __launch_bounds__(kThreads) k_scan_spine(unsigned long long* partial, uint64_t nb,
                                                         unsigned long long* total_out) {
  __shared__ unsigned long long tmp[kThreads / 32 + 1];
  unsigned long long carry = 0;
  for (uint64_t c = 0; c < nb; c += kThreads) {
    uint64_t i = c + threadIdx.x;
    unsigned long long v = (i < nb) ? partial[i] : 0ull;
    unsigned long long tot;
    unsigned long long ex = block_excl_u64(v, tmp, &tot);
    if (i < nb) partial[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

template <typename In, typename Out>
__global__ void __launch_bounds__(kThreads) k_scan_down(In in, uint64_t n, const unsigned long long* partial,
                                                        const unsigned long long* total, Out* out,
                                                        int write_last, uint32_t stride) {
  __shared__ unsigned long long tmp[kThreads / 32 + 1];
  const uint64_t base = (uint64_t)blockIdx.x * kTile;
  unsigned long long carry = partial[blockIdx.x];
  for (int r = 0; r < kItems; ++r) {
    uint64_t i = base + (uint64_t)r * kThreads + threadIdx.x;
    if (base + (uint64_t)r * kThreads >= n) break;  // uniform across the block
    unsigned long long v = (i < n) ? in(i) : 0ull;
    unsigned long long tot;
    unsigned long long ex = block_excl_u64(v, tmp, &tot);
    if (i < n) out[i * stride] = (Out)(carry + ex);
    carry += tot;
  }
  if (write_last && blockIdx.x == 0 && threadIdx.x == 0) out[n * stride] = (Out)(*total);
}

template <typename Out>
__global__ void k_store_total(const unsigned long long* total, Out* dst) {
  *dst = (Out)(*total);
}

// Exclusive scan of in(0..n-1) into out[i * stride] (and out[n * stride] =
// total if write_last; *total_dst = total if not null).
template <typename In, typename Out>
cudaError_t scan_impl(Launcher* L, In in, uint64_t n, Out* out, int write_last, Out* total_dst, void* temp,
                      cudaStream_t s, uint32_t stride = 1) {
  uint64_t nb = (n + kTile - 1) / kTile;
  if (nb == 0) nb = 1;
  unsigned long long* partial = (unsigned long long*)temp;
  unsigned long long* total = partial + nb;
  cudaError_t e;
  if ((e = launch_begin(L, "scan_reduce")) != cudaSuccess) return e;
  k_scan_reduce<In><<<(unsigned)nb, kThreads, 0, s>>>(in, n, partial);
  if ((e = launch_end(L, "scan_reduce")) != cudaSuccess) return e;
  if ((e = launch_begin(L, "scan_spine")) != cudaSuccess) return e;
  k_scan_spine<<<1, kThreads, 0, s>>>(partial, nb, total);
  if ((e = launch_end(L, "scan_spine")) != cudaSuccess) return e;
  if ((e = launch_begin(L, "scan_down")) != cudaSuccess) return e;
  k_scan_down<In, Out><<<(unsigned)nb, kThreads, 0, s>>>(in, n, partial, total, out, write_last, stride);
  if ((e = launch_end(L, "scan_down")) != cudaSuccess) return e;
  if (total_dst) {
    if ((e = launch_begin(L, "scan_total")) != cudaSuccess) return e;
    k_store_total<Out><<<1, 1, 0, s>>>(total, total_dst);
    if ((e = launch_end(L, "scan_total")) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

size_t scan_temp_bytes(uint64_t n) {
  uint64_t nb = (n + kTile - 1) / kTile;
  if (nb == 0) nb = 1;
  return (size_t)(nb + 1) * sizeof(unsigned long long);
}

cudaError_t scan_dict_blocks(Launcher* L, uint32_t* dict, uint64_t n_blocks, uint32_t* total, void* temp,
                             cudaStream_t s) {
  // in() reads words 1..7 of a block, out writes its word 0: no overlap
  return scan_impl<DictIn, uint32_t>(L, DictIn{dict}, n_blocks, dict, 0, total, temp, s, 8u);
}

cudaError_t scan_u32(Launcher* L, const uint32_t* in, uint64_t n, uint32_t* out_excl_np1, void* temp,
                     cudaStream_t s) {
  return scan_impl<U32In, uint32_t>(L, U32In{in}, n, out_excl_np1, 1, nullptr, temp, s);
}

cudaError_t scan_u32_to_u64(Launcher* L, const uint32_t* in, uint64_t n, unsigned long long* out_excl_np1,
                            void* temp, cudaStream_t s) {
  return scan_impl<U32In, unsigned long long>(L, U32In{in}, n, out_excl_np1, 1, nullptr, temp, s);
}

}  // namespace pdg
