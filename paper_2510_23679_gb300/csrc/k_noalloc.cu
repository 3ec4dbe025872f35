// k_noalloc.cu -- Best Hits of one genome pair without any device allocation.
//
// pd_best_hits_noalloc runs the same sum-min / Best Hit kernels as
// pd_best_hits (k_summin.cu), but every temporary buffer -- counters, the per-
// row offsets and lengths, the unordered hit list, the lists of queries
// handed to the larger tiers, the global-memory tables of the last tier and
// the prefix-sum scratch -- is carved out of one fixed array in device memory
// that this file declares, and the CSR result goes straight into buffers the
// caller owns.  It is for callers that cannot allocate device memory while
// they run: a process whose device memory is all owned by an external pool or
// memory manager, or a latency-critical loop where an allocation could block
// or fail at the worst moment.  They set up profiles and output buffers once
// and then query pairs with no allocation on the path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "pd.h"
#include "pd_internal.cuh"

#define PD_API extern "C" __attribute__((visibility("default")))

namespace {

// The scratch of every call on every device (each device that loads the
// library holds its own copy until the process exits).
static __device__ __align__(256) unsigned char g_noalloc_scratch[PD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
constexpr uint32_t kGlobalTierBlocks = 8;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (which must be current).
// In host code the array's name only stands in for the symbol, so the address
// is looked up once per device and cached.  The cached address belongs to the
// device's primary context: it stays valid until that context is destroyed
// (cudaDeviceReset), after which the library must be loaded again.
cudaError_t scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = (unsigned char*)g_scratch_addr[device];
  return cudaSuccess;
}

// Bump allocator over the scratch array (256-byte aligned pieces).
struct Carve {
  unsigned char* base;
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    const size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
    if (used + bytes > (size_t)PD_NOALLOC_SCRATCH_BYTES) return nullptr;
    T* p = (T*)(base + used);
    used += bytes;
    return p;
  }
};

// True if p is device (or managed) memory that kernels on `device` address.
bool is_device_ptr(const void* p, int device) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace

namespace {

pd_status noalloc_impl(pd_ctx* ctx, const pd_profiles* prof, uint32_t gi, uint32_t gj, int64_t* row_ptr,
                       int32_t* cols, uint32_t* s, uint64_t capacity, uint64_t* n_hits) {
  using namespace pdg;
  CtxView cv;
  if (!ctx_view(ctx, &cv)) return PD_ERR_ARG;
  const ProfilesView* P = profiles_view(prof);
  if (!P) return ctx_fail(ctx, PD_ERR_ARG, "null profiles");
  if (gi >= P->n_genomes || gj >= P->n_genomes || gi == gj)
    return ctx_fail(ctx, PD_ERR_ARG, "genome indices must be distinct and < n_genomes");
  const uint32_t qa0 = (uint32_t)profiles_genome_start(prof, gi);
  const uint32_t nA = (uint32_t)profiles_genome_start(prof, gi + 1) - qa0;
  const uint32_t ta0 = (uint32_t)profiles_genome_start(prof, gj);
  const uint32_t ta1 = (uint32_t)profiles_genome_start(prof, gj + 1);
  if (nA > PD_NOALLOC_MAX_ROWS)
    return ctx_fail(ctx, PD_ERR_ARG, "pd_best_hits_noalloc: query genome has more than PD_NOALLOC_MAX_ROWS genes");
  if (ta1 - ta0 > PD_NOALLOC_MAX_TARGETS)
    return ctx_fail(ctx, PD_ERR_ARG,
                    "pd_best_hits_noalloc: target genome has more than PD_NOALLOC_MAX_TARGETS genes");
  if (!is_device_ptr(row_ptr, cv.device) ||
      (capacity > 0 && (!is_device_ptr(cols, cv.device) || !is_device_ptr(s, cv.device))))
    return ctx_fail(ctx, PD_ERR_ARG,
                    "pd_best_hits_noalloc: row_ptr, cols and s must be device memory of the context's device");
  cudaError_t e = cudaSetDevice(cv.device);
  unsigned char* scratch = nullptr;
  if (e == cudaSuccess) e = scratch_address(cv.device, &scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(ctx, PD_ERR_CUDA, "pd_best_hits_noalloc: scratch array address unavailable");
  }

  // ---- layout of this call in the scratch array
  Carve cv_mem{scratch};
  const uint32_t rows = std::max<uint32_t>(nA, 1);
  const uint32_t targets = std::max<uint32_t>(ta1 - ta0, 2);
  unsigned long long* counters = cv_mem.take<unsigned long long>(4);
  unsigned long long* row_off = cv_mem.take<unsigned long long>(rows);
  uint32_t* row_len = cv_mem.take<uint32_t>(rows);
  uint32_t* def1 = cv_mem.take<uint32_t>(rows);
  uint32_t* def2 = cv_mem.take<uint32_t>(rows);
  uint32_t* out_b = cv_mem.take<uint32_t>(PD_NOALLOC_MAX_HITS);
  uint32_t* out_s = cv_mem.take<uint32_t>(PD_NOALLOC_MAX_HITS);
  void* scan_tmp = cv_mem.take<unsigned char>(scan_temp_bytes((uint64_t)nA + 1));
  BigScratch B;
  B.cap = std::max<uint32_t>(next_pow2(4 * targets), 256);  // load <= 1/4: short probe chains
  B.out_cap = next_pow2(targets);
  B.keys = cv_mem.take<uint32_t>((size_t)B.cap * kGlobalTierBlocks);
  B.vals = cv_mem.take<uint32_t>((size_t)B.cap * kGlobalTierBlocks);
  B.used = cv_mem.take<uint32_t>((size_t)B.cap * kGlobalTierBlocks);
  B.out = cv_mem.take<unsigned long long>((size_t)B.out_cap * kGlobalTierBlocks);
  if (!counters || !row_off || !row_len || !def1 || !def2 || !out_b || !out_s || !scan_tmp || !B.keys || !B.vals ||
      !B.used || !B.out)
    return ctx_fail(ctx, PD_ERR_INTERNAL, "pd_best_hits_noalloc: scratch layout exceeds the array");

  // ---- sum-min and Best Hits of G_gi against G_gj (shared tiers, then the
  // global tier inside the scratch array if any query needs it)
  cudaStream_t st = cv.stream;
  Launcher* L = cv.launcher;
  QuerySet Q{};
  Q.all_pairs = 0;
  Q.qa0 = qa0;
  Q.nA = nA;
  Q.ta0 = ta0;
  Q.ta1 = ta1;
  Q.n_queries = nA;
  HitsOut O;
  O.out_b = out_b;
  O.out_s = out_s;
  O.out_cap = PD_NOALLOC_MAX_HITS;
  O.cursor = counters + 0;
  O.walked = counters + 1;
  O.n_def1 = (uint32_t*)(counters + 2);
  O.n_def2 = (uint32_t*)(counters + 3);
  O.row_off = row_off;
  O.row_len = row_len;
  O.def1 = def1;
  O.def2 = def2;
  unsigned long long h[4] = {0, 0, 0, 0};
  if ((e = cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned long long), st)) != cudaSuccess) return ctx_fail(ctx, PD_ERR_CUDA, cudaGetErrorString(e));
  if ((e = cudaMemsetAsync(row_len, 0, sizeof(uint32_t) * rows, st)) != cudaSuccess) return ctx_fail(ctx, PD_ERR_CUDA, cudaGetErrorString(e));
  if (nA) {
    if ((e = run_summin_tiers(L, *P, Q, O, cv.d_err, false, st)) != cudaSuccess)
      return ctx_fail(ctx, PD_ERR_CUDA, cudaGetErrorString(e));
    if ((e = cudaMemcpyAsync(h, counters, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return ctx_fail(ctx, PD_ERR_CUDA, cudaGetErrorString(e));
    if (h[3] > 0) {
      if ((e = run_summin_global(L, *P, Q, O, B, std::min<uint32_t>((uint32_t)h[3], kGlobalTierBlocks), cv.d_err,
                                 false, st)) != cudaSuccess)
        return ctx_fail(ctx, PD_ERR_CUDA, cudaGetErrorString(e));
      if ((e = cudaMemcpyAsync(h, counters, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return ctx_fail(ctx, PD_ERR_CUDA, cudaGetErrorString(e));
    }
    // device-side errors (the pinned mirror belongs to the context)
    if ((e = cudaMemcpyAsync(cv.h_err, cv.d_err, sizeof(DevErr), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return ctx_fail(ctx, PD_ERR_CUDA, cudaGetErrorString(e));
    if (cv.h_err->code != 0) {
      const int code = cv.h_err->code;
      cudaMemsetAsync(cv.d_err, 0, sizeof(DevErr), st);
      return ctx_fail(ctx, (pd_status)code, "pd_best_hits_noalloc: device reported an error");
    }
  }
  const uint64_t total = h[0];
  if (n_hits) *n_hits = total;
  if (total > PD_NOALLOC_MAX_HITS)
    return ctx_fail(ctx, PD_ERR_BUDGET, "pd_best_hits_noalloc: more than PD_NOALLOC_MAX_HITS Best Hit entries");
  if (total > capacity)
    return ctx_fail(ctx, PD_ERR_ARG, "pd_best_hits_noalloc: cols/s hold fewer entries than *n_hits");

  // ---- CSR into the caller's buffers
  if ((e = scan_u32_to_u64(L, row_len, nA, (unsigned long long*)row_ptr, scan_tmp, st)) != cudaSuccess)
    return ctx_fail(ctx, PD_ERR_CUDA, cudaGetErrorString(e));
  if (nA && total) {
    if ((e = run_gather_rows(L, nA, row_off, row_len, (const unsigned long long*)row_ptr, out_b, out_s, ta0, cols,
                             s, st)) != cudaSuccess)
      return ctx_fail(ctx, PD_ERR_CUDA, cudaGetErrorString(e));
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return ctx_fail(ctx, PD_ERR_CUDA, cudaGetErrorString(e));
  return PD_OK;
}

}  // namespace

PD_API pd_status pd_best_hits_noalloc(pd_ctx* ctx, const pd_profiles* prof, uint32_t gi, uint32_t gj,
                                      int64_t* row_ptr, int32_t* cols, uint32_t* s, uint64_t capacity,
                                      uint64_t* n_hits) {
  if (!ctx || !prof) return PD_ERR_ARG;
  try {
    // no per-kernel timing events for this call (creating them would allocate)
    const bool timing = pdg::ctx_swap_timing(ctx, false);
    const pd_status st = noalloc_impl(ctx, prof, gi, gj, row_ptr, cols, s, capacity, n_hits);
    pdg::ctx_swap_timing(ctx, timing);
    return st;
  } catch (...) {
    return pdg::ctx_fail(ctx, PD_ERR_INTERNAL, "exception in pd_best_hits_noalloc");
  }
}
