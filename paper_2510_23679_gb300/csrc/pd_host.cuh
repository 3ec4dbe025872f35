// pd_host.cuh -- host-side pieces shared by the translation units that
// implement the C ABI (pd_api.cu, pd_batch.cu): the context, the device
// buffer type that allocates through the context's hooks, error helpers,
// the handle types, and the internal entry points one unit calls in another.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pd.h"
#include "pd_internal.cuh"

#define PD_API extern "C" __attribute__((visibility("default")))

// A named range around one phase of a call (profile build, Best Hits, BBH,
// a served tick), visible to profilers as an NVTX range; without a profiler
// attached it costs a pointer test.
struct PhaseRange {
  explicit PhaseRange(const char* name) { nvtxRangePushA(name); }
  ~PhaseRange() { nvtxRangePop(); }
  PhaseRange(const PhaseRange&) = delete;
  PhaseRange& operator=(const PhaseRange&) = delete;
};

struct pd_ctx;

namespace pdg {

struct Launcher {
  pd_ctx* ctx;
};

}  // namespace pdg

struct PendingTiming {
  std::string name;
  cudaEvent_t start, stop;
};

struct pd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  pd_alloc_fn alloc = nullptr;
  pd_free_fn free_fn = nullptr;
  void* user = nullptr;
  std::string err;
  uint64_t launches = 0;
  bool timing = false;
  bool symmetric = true;  // pd_best_hits_all walks each genome pair from one side (pd_ctx_set_symmetric)
  uint32_t walk = PD_WALK_AUTO;  // posting walk of the sum-min kernel (pd_ctx_set_walk)
  std::string timing_filter;  // empty: time every kernel; else only launches of this name
  std::vector<PendingTiming> pending;
  std::vector<cudaEvent_t> event_pool;
  std::map<std::string, std::pair<double, uint64_t>> kernel_ms;
  pdg::Launcher L{nullptr};
  pdg::DevErr* d_err = nullptr;  // device error block
  pdg::DevErr* h_err = nullptr;  // pinned host mirror
  // pinned host words the profile build reads back after its dictionary pass
  unsigned long long* h_build = nullptr;  // [8]
  int32_t* h_genome_ptr = nullptr;        // [PD_MAX_GENOMES + 1]
  cudaMemPool_t pool = nullptr;  // without hooks: allocate from this pool (null: the device's default pool)
  bool own_pool = false;         // the pool was created by (and is destroyed with) this context
  uint64_t pool_bytes = 0;       // bytes currently allocated through this context (pool allocations only)
};

// ------------------------------------------------------------------ helpers
namespace pdh {

using pdg::DevErr;

inline pd_status fail(pd_ctx* c, pd_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

inline pd_status fail_cuda(pd_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return fail(c, PD_ERR_CUDA, m);
}

#define CK(expr)                                      \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return fail_cuda(c, e_, #expr); \
  } while (0)

// Device buffer owned through the context's allocator.
struct Buf {
  pd_ctx* c = nullptr;
  void* p = nullptr;
  size_t n = 0;
  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  Buf(Buf&& o) noexcept : c(o.c), p(o.p), n(o.n) { o.p = nullptr; }
  Buf& operator=(Buf&& o) noexcept {
    if (this != &o) {
      release();
      c = o.c;
      p = o.p;
      n = o.n;
      o.p = nullptr;
    }
    return *this;
  }
  ~Buf() { release(); }
  bool alloc(pd_ctx* ctx, size_t bytes) {
    release();
    c = ctx;
    n = (std::max<size_t>(bytes, 16) + 255) & ~(size_t)255;
    if (c->alloc) {
      p = c->alloc(n, (void*)c->stream, c->user);
    } else if (c->pool) {
      if (cudaMallocFromPoolAsync(&p, n, c->pool, c->stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
      } else {
        c->pool_bytes += n;
      }
    } else if (cudaMallocAsync(&p, n, c->stream) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return p != nullptr;
  }
  void release() {
    if (p && c) {
      if (c->free_fn) {
        c->free_fn(p, n, (void*)c->stream, c->user);
      } else {
        cudaFreeAsync(p, c->stream);
        if (c->pool) c->pool_bytes -= n;
      }
    }
    p = nullptr;
  }
  template <typename T>
  T* as() const {
    return (T*)p;
  }
};

#define ALLOC(buf, bytes)                                                                        \
  do {                                                                                           \
    if (!(buf).alloc(c, (bytes))) return fail(c, PD_ERR_OOM, "device allocation of " +           \
                                                             std::to_string((size_t)(bytes)) +   \
                                                             " bytes failed (" #buf ")");        \
  } while (0)

inline bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline uint32_t bits_for(uint32_t max_value) {
  uint32_t b = 1;
  while (b < 32 && (max_value >> b) != 0) ++b;
  return b;
}

inline uint64_t pow_u64(uint64_t b, int e) {
  uint64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// Reads the device error block; returns PD_OK or the recorded error.
inline pd_status check_dev_err(pd_ctx* c) {
  CK(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(DevErr), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (c->h_err->code != 0) {
    const int code = c->h_err->code;
    const unsigned long long det = c->h_err->detail;
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(DevErr), c->stream));
    if (code == PD_ERR_ALPHABET)
      return fail(c, PD_ERR_ALPHABET, "residue at offset " + std::to_string(det) +
                                          " is not a letter of the alphabet (ACDEFGHIKLMNPQRSTVWY or ACGT)");
    return fail(c, (pd_status)code, "device reported error " + std::to_string(code) + " (detail " +
                                        std::to_string(det) + ")");
  }
  return PD_OK;
}

// Copy `bytes` from a device buffer to a caller pointer (host or device).
inline pd_status copy_out(pd_ctx* c, void* dst, const void* src, size_t bytes) {
  if (!dst || bytes == 0) return PD_OK;
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
  return PD_OK;
}

}  // namespace pdh

// ------------------------------------------------------------------ handles
using pdh::Buf;

struct pd_profiles {
  pd_ctx* ctx = nullptr;
  pdg::ProfilesView view{};
  pd_profiles_info info{};
  Buf genome_ptr, La, win_off, mv_n, mv_id, mv_cnt, mv_post, mv_plen, gene_genome, ginfo, dict, post_ptr,
      post, order;
  std::vector<int32_t> h_genome_ptr;
};

struct pd_hits {
  pd_ctx* ctx = nullptr;
  int all_pairs = 0;
  int paralog = 0;  // within-genome Best Hits (rows = all genes)
  uint32_t n_rows = 0, row_base = 0, col_base = 0;
  uint32_t nA = 0, qa0 = 0, qb0 = 0;  // pair form with both directions (internal)
  uint64_t n_hits = 0, walked = 0;
  uint32_t n_deferred = 0;
  Buf row_off, row_len, out_b, out_s;
  // the symmetric all-pairs form finds the BBH pairs with the rows, and its
  // rows are already one CSR: row_off holds n_rows + 1 offsets into
  // out_b / out_s, in row order
  bool has_bbh = false;
  bool csr = false;
  uint64_t n_bbh = 0;
  Buf bbh_a, bbh_b;
};

struct pd_bbh_set {
  pd_ctx* ctx = nullptr;
  uint64_t n = 0;
  Buf a, b;
};


// Genes profiled against another dataset's dictionary (external queries):
// their vectors hold only k-mers that dataset contains, with posting ranges
// into its index, while La counts every window.
struct QueryProfiles {
  uint32_t n_genes = 0;
  Buf win_off, mv_n, mv_id, mv_cnt, mv_post, mv_plen, La;
};

// ------------------------------------------------------------------ internal entry points (pd_api.cu)
namespace pdh {

// Profiles of n_genes genes (residues on the device, gene_ptr on the host from
// 0) against the dictionary and index of P; windows with letters outside the
// alphabet must have been rejected by the caller.
pd_status query_profiles_impl(pd_ctx* c, const pd_profiles* P, const uint8_t* residues_dev, const int64_t* gene_ptr,
                              uint32_t n_genes, QueryProfiles* out);
// P's view with the external query arrays of Qp.
pdg::ProfilesView external_view(const pd_profiles* P, const QueryProfiles& Qp);
// run_hits on an explicit view (external queries).
pd_status run_hits_view(pd_ctx* c, const pdg::ProfilesView& v, const pdg::QuerySet& Q, pd_hits* H,
                        uint32_t genomes_per_query);

// Profiles of a dataset; genome_seg (host, per genome, or null) gives each
// segment its own k-mer namespace.  gene_src (device, per gene, or null):
// gene g starts at residues + gene_src[g] instead of residues + gene_ptr[g];
// gene_ptr then gives only the lengths, and residues must be a device pointer.
pd_status build_profiles_impl(pd_ctx* c, const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr,
                              uint32_t n_genes, const int32_t* genome_ptr, uint32_t n_genomes, int k,
                              const uint32_t* genome_seg, pd_profiles** out, const int64_t* gene_src = nullptr,
                              int alphabet = PD_ALPHABET_AMINO, int length_buckets = 1);
// Sum-min + Best Hits of the query set Q into H (all tiers, output sized
// exactly).  genomes_per_query (0 = n_genomes - 1) bounds the genomes one
// query can hit; it only sizes the first output allocation.
pd_status run_hits(pd_ctx* c, const pd_profiles* P, const pdg::QuerySet& Q, bool emit_all, pd_hits* H,
                   uint32_t genomes_per_query = 0);
// Mutual Best Hits of the rows R into S.
pd_status bbh_impl(pd_ctx* c, const pdg::BbhRows& R, uint64_t n_hit_slots, uint32_t a_base, uint32_t b_base,
                   pd_bbh_set* S);

}  // namespace pdh
