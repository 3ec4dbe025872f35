// pd_api.cu -- host side of the C ABI declared in include/pd.h.
//
// Orchestrates the kernels of k_profiles.cu, k_summin.cu, k_bbh.cu and
// k_scan.cu on the context's stream, owns device memory through the
// context's allocator hooks, and turns every failure into a pd_status with a
// message (no exception crosses the ABI).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "pd.h"
#include "pd_host.cuh"
#include "pd_internal.cuh"

using namespace pdh;

// ------------------------------------------------------------------ launches
namespace pdg {

static cudaEvent_t take_event(pd_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

cudaError_t launch_begin(Launcher* L, const char* name) {
  pd_ctx* c = L->ctx;
  if (c->timing && (c->timing_filter.empty() || c->timing_filter == name)) {
    PendingTiming t{name, take_event(c), take_event(c)};
    if (!t.start || !t.stop) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaEventRecord(t.start, c->stream);
    if (e != cudaSuccess) return e;
    c->pending.push_back(t);
  }
  return cudaSuccess;
}

cudaError_t launch_end(Launcher* L, const char* name) {
  pd_ctx* c = L->ctx;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  c->launches += 1;
  if (c->timing && !c->pending.empty() && c->pending.back().name == name)
    return cudaEventRecord(c->pending.back().stop, c->stream);
  return cudaSuccess;
}

}  // namespace pdg

// ------------------------------------------------------------------ internal accessors
// Read-only views of the handles for other translation units of the library
// (the allocation-free entry point of k_noalloc.cu).
namespace pdg {

bool ctx_view(pd_ctx* c, CtxView* v) {
  if (!c || !v) return false;
  v->stream = c->stream;
  v->device = c->device;
  v->d_err = c->d_err;
  v->h_err = c->h_err;
  v->launcher = &c->L;
  return true;
}

bool ctx_swap_timing(pd_ctx* c, bool on) {
  const bool was = c->timing;
  c->timing = on;
  return was;
}

pd_status ctx_fail(pd_ctx* c, pd_status st, const char* msg) {
  if (c) c->err = msg;
  return st;
}

const ProfilesView* profiles_view(const pd_profiles* P) { return P ? &P->view : nullptr; }

int32_t profiles_genome_start(const pd_profiles* P, uint32_t g) { return P->h_genome_ptr[g]; }

}  // namespace pdg

// ------------------------------------------------------------------ context
PD_API pd_status pd_ctx_create(int device, void* cuda_stream, pd_alloc_fn alloc, pd_free_fn free_fn, void* user,
                               pd_ctx** out) {
  if (!out) return PD_ERR_ARG;
  *out = nullptr;
  if ((alloc == nullptr) != (free_fn == nullptr)) return PD_ERR_ARG;
  pd_ctx* c = nullptr;
  try {
    c = new pd_ctx();
  } catch (...) {
    return PD_ERR_OOM;
  }
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  c->alloc = alloc;
  c->free_fn = free_fn;
  c->user = user;
  c->L.ctx = c;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(DevErr));
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_err, sizeof(DevErr));
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_build, 8 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_genome_ptr, sizeof(int32_t) * (PD_MAX_GENOMES + 1));
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(DevErr));
  if (e == cudaSuccess && !alloc) {
    // Without hooks the context allocates from a pool of its own that keeps
    // freed memory for reuse (no release back to the driver between calls).
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    e = cudaMemPoolCreate(&c->pool, &props);
    if (e == cudaSuccess) {
      c->own_pool = true;
      uint64_t keep = ~0ull;
      e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (c->d_err) cudaFree(c->d_err);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->h_build) cudaFreeHost(c->h_build);
    if (c->h_genome_ptr) cudaFreeHost(c->h_genome_ptr);
    if (c->own_pool) cudaMemPoolDestroy(c->pool);
    delete c;
    return PD_ERR_CUDA;
  }
  *out = c;
  return PD_OK;
}

PD_API void pd_ctx_destroy(pd_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (auto& t : c->pending) {
    cudaEventDestroy(t.start);
    cudaEventDestroy(t.stop);
  }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  cudaFree(c->d_err);
  cudaFreeHost(c->h_err);
  cudaFreeHost(c->h_build);
  cudaFreeHost(c->h_genome_ptr);
  // allocations still held by handles keep the pool alive until they are freed
  if (c->own_pool) cudaMemPoolDestroy(c->pool);
  delete c;
}

PD_API pd_status pd_ctx_set_stream(pd_ctx* c, void* cuda_stream) {
  if (!c) return PD_ERR_ARG;
  c->stream = (cudaStream_t)cuda_stream;
  return PD_OK;
}

PD_API const char* pd_last_error(const pd_ctx* c) { return c ? c->err.c_str() : "null context"; }

PD_API uint64_t pd_ctx_launch_count(const pd_ctx* c) { return c ? c->launches : 0; }

PD_API pd_status pd_ctx_set_symmetric(pd_ctx* c, int enable) {
  if (!c) return PD_ERR_ARG;
  c->symmetric = enable != 0;
  return PD_OK;
}

PD_API pd_status pd_ctx_set_walk(pd_ctx* c, uint32_t mode) {
  if (!c) return PD_ERR_ARG;
  if (mode > PD_WALK_WARP) return fail(c, PD_ERR_ARG, "unknown walk mode");
  c->walk = mode;
  return PD_OK;
}

PD_API pd_status pd_ctx_set_timing(pd_ctx* c, int enable) {
  if (!c) return PD_ERR_ARG;
  c->timing = enable != 0;
  return PD_OK;
}

PD_API pd_status pd_ctx_set_timing_filter(pd_ctx* c, const char* name) {
  if (!c) return PD_ERR_ARG;
  try {
    c->timing_filter = name ? name : "";
  } catch (...) {
    return fail(c, PD_ERR_OOM, "out of host memory");
  }
  return PD_OK;
}

static pd_status drain_timing(pd_ctx* c) {
  CK(cudaStreamSynchronize(c->stream));
  for (auto& t : c->pending) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, t.start, t.stop));
    auto& acc = c->kernel_ms[t.name];
    acc.first += ms;
    acc.second += 1;
    c->event_pool.push_back(t.start);
    c->event_pool.push_back(t.stop);
  }
  c->pending.clear();
  return PD_OK;
}

PD_API pd_status pd_ctx_kernel_time(pd_ctx* c, const char* name, double* ms, uint64_t* launches) {
  if (!c) return PD_ERR_ARG;
  try {
    pd_status st = drain_timing(c);
    if (st != PD_OK) return st;
    double t = 0;
    uint64_t n = 0;
    for (auto& kv : c->kernel_ms) {
      if (name == nullptr || kv.first == name) {
        t += kv.second.first;
        n += kv.second.second;
      }
    }
    if (ms) *ms = t;
    if (launches) *launches = n;
    return PD_OK;
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_ctx_kernel_time");
  }
}

PD_API pd_status pd_ctx_reset_timing(pd_ctx* c) {
  if (!c) return PD_ERR_ARG;
  pd_status st = drain_timing(c);
  c->kernel_ms.clear();
  return st;
}

PD_API int pd_choose_k(uint64_t total, int alphabet) {
  if (alphabet < 2) return -1;
  int k = 1;
  unsigned __int128 p = (unsigned __int128)alphabet;
  while (p < total) {
    p *= (unsigned)alphabet;
    ++k;
  }
  return k;
}

// ------------------------------------------------------------------ profiles
// Most codes a segmented dataset's dictionary may cover (segments x 20^k): one
// bit each, 4 GiB of bits (4.6 GiB of rank blocks).
static constexpr uint64_t kMaxDictCodes = (uint64_t)32 << 30;

pd_status pdh::build_profiles_impl(pd_ctx* c, const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr,
                                     uint32_t n_genes, const int32_t* genome_ptr, uint32_t n_genomes, int k,
                                     const uint32_t* genome_seg, pd_profiles** out, const int64_t* gene_src,
                                     int alphabet, int length_buckets) {
  PhaseRange range_("pd: profiles");
  if (alphabet != PD_ALPHABET_AMINO && alphabet != PD_ALPHABET_NUCLEOTIDE)
    return fail(c, PD_ERR_ARG, "alphabet must be 20 (amino acids) or 4 (nucleotides)");
  const int max_k = alphabet == PD_ALPHABET_AMINO ? PD_MAX_K : PD_MAX_K_NUCLEOTIDE;
  if (k < 1 || k > max_k) return fail(c, PD_ERR_K_RANGE, "k must be in [1, " + std::to_string(max_k) + "]");
  if (!gene_ptr || !genome_ptr || (n_res > 0 && !residues))
    return fail(c, PD_ERR_ARG, "null residues, gene_ptr or genome_ptr");
  if (n_genomes < 1 || n_genomes > PD_MAX_GENOMES)
    return fail(c, PD_ERR_ARG, "n_genomes must be in [1, " + std::to_string(PD_MAX_GENOMES) + "]");
  if (n_genes > 0x7FFFFFFFu) return fail(c, PD_ERR_ARG, "too many genes");
  if (n_genes == 0 && n_res != 0 && !gene_src) return fail(c, PD_ERR_ARG, "residues without genes");
  CK(cudaSetDevice(c->device));

  // ---- genome offsets on the host (small; checked before any kernel reads them,
  // except on the non-segmented path with device offsets, where the checks
  // come after the dictionary pass and before the first kernel that uses them)
  std::vector<int32_t> hgn(n_genomes + 1);
  const bool gp_dev = is_device_ptr(gene_ptr), gn_dev = is_device_ptr(genome_ptr);
  const bool early_genomes = !gn_dev || genome_seg;
  if (gn_dev) {
    CK(cudaMemcpyAsync(c->h_genome_ptr, genome_ptr, sizeof(int32_t) * (n_genomes + 1), cudaMemcpyDeviceToHost,
                       c->stream));
    if (early_genomes) CK(cudaStreamSynchronize(c->stream));
  } else {
    std::copy(genome_ptr, genome_ptr + n_genomes + 1, c->h_genome_ptr);
  }
  auto check_genomes = [&]() -> pd_status {
    std::copy(c->h_genome_ptr, c->h_genome_ptr + n_genomes + 1, hgn.begin());
    if (hgn[0] != 0 || (uint32_t)hgn[n_genomes] != n_genes)
      return fail(c, PD_ERR_ARG, "genome_ptr must run from 0 to n_genes");
    for (uint32_t i = 0; i < n_genomes; ++i)
      if (hgn[i + 1] < hgn[i]) return fail(c, PD_ERR_ARG, "genome_ptr is decreasing at " + std::to_string(i));
    return PD_OK;
  };
  if (early_genomes) {
    pd_status st0 = check_genomes();
    if (st0 != PD_OK) return st0;
  }

  pd_profiles* P = new pd_profiles();
  P->ctx = c;
  std::unique_ptr<pd_profiles> guard(P);
  const uint64_t n_codes = pow_u64((uint64_t)alphabet, k);
  uint64_t n_seg = 1;
  std::vector<unsigned long long> code_base;
  if (genome_seg) {
    code_base.resize(n_genomes);
    for (uint32_t i = 0; i < n_genomes; ++i) {
      if (genome_seg[i] >= n_genomes) return fail(c, PD_ERR_ARG, "genome_seg values must be < n_genomes");
      n_seg = std::max<uint64_t>(n_seg, (uint64_t)genome_seg[i] + 1);
      code_base[i] = (unsigned long long)genome_seg[i] * n_codes;
    }
    if (n_seg * n_codes > kMaxDictCodes)
      return fail(c, PD_ERR_BUDGET, "segments x 20^k exceed the dictionary limit (" +
                                        std::to_string(kMaxDictCodes >> 30) + " Gi codes)");
  }
  const uint64_t n_dict = pdg::dict_blocks(n_seg * n_codes);
  const size_t G1 = std::max<uint32_t>(n_genes, 1);
  pdg::Launcher* L = &c->L;

  // ---- inputs on the device
  Buf d_res, d_gene_ptr, d_mid, d_long, d_long_off, d_long_scratch, tmp, d_counts, minhash, d_code_base;
  const uint8_t* res_dev = residues;
  const int64_t* gp_devp = gene_ptr;
  if (n_res > 0 && !is_device_ptr(residues)) {
    ALLOC(d_res, n_res);
    CK(cudaMemcpyAsync(d_res.p, residues, n_res, cudaMemcpyHostToDevice, c->stream));
    res_dev = d_res.as<uint8_t>();
  }
  if (!gp_dev) {
    ALLOC(d_gene_ptr, sizeof(int64_t) * (n_genes + 1));
    CK(cudaMemcpyAsync(d_gene_ptr.p, gene_ptr, sizeof(int64_t) * (n_genes + 1), cudaMemcpyHostToDevice,
                       c->stream));
    gp_devp = d_gene_ptr.as<int64_t>();
  }
  ALLOC(P->genome_ptr, sizeof(int32_t) * (n_genomes + 1));
  ALLOC(P->La, sizeof(uint32_t) * G1);
  ALLOC(P->win_off, sizeof(uint32_t) * (n_genes + 1));
  ALLOC(P->gene_genome, sizeof(uint16_t) * G1);
  ALLOC(P->ginfo, sizeof(uint32_t) * G1);
  CK(cudaMemcpyAsync(P->genome_ptr.p, genome_ptr, sizeof(int32_t) * (n_genomes + 1), cudaMemcpyDefault, c->stream));

  // ---- window counts, window offsets and the gene classes, on the device
  Buf d_win64, d_gtmp, d_wcount;
  ALLOC(d_mid, sizeof(uint32_t) * G1);
  ALLOC(d_long, sizeof(uint32_t) * G1);
  ALLOC(d_long_off, sizeof(unsigned long long) * G1);
  ALLOC(d_win64, sizeof(unsigned long long) * (n_genes + 1));
  ALLOC(d_gtmp, pdg::scan_temp_bytes(n_genes + 1) + 64);
  ALLOC(d_wcount, 4 * sizeof(unsigned long long));  // [n_mid, n_long] (u32), long_total (u64)
  CK(cudaMemsetAsync(d_wcount.p, 0, 4 * sizeof(unsigned long long), c->stream));
  unsigned long long* wcount64 = d_wcount.as<unsigned long long>();
  if (n_genes)
    CK(pdg::run_gene_windows(L, gp_devp, n_genes, n_res, gene_src ? 0 : 1, k, P->La.as<uint32_t>(),
                             d_mid.as<uint32_t>(), d_long.as<uint32_t>(), d_long_off.as<unsigned long long>(),
                             (uint32_t*)wcount64, wcount64 + 1, c->d_err, c->stream));
  CK(pdg::scan_u32_to_u64(L, P->La.as<uint32_t>(), n_genes, d_win64.as<unsigned long long>(), d_gtmp.p, c->stream));
  CK(pdg::run_narrow_u64(L, d_win64.as<unsigned long long>(), n_genes + 1, P->win_off.as<uint32_t>(), c->stream));
  if (early_genomes)
    CK(pdg::run_gene_info(L, P->genome_ptr.as<int32_t>(), n_genomes, P->La.as<uint32_t>(),
                          P->gene_genome.as<uint16_t>(), P->ginfo.as<uint32_t>(), c->stream));

  if (genome_seg) {
    ALLOC(d_code_base, sizeof(unsigned long long) * n_genomes);
    CK(cudaMemcpyAsync(d_code_base.p, code_base.data(), sizeof(unsigned long long) * n_genomes,
                       cudaMemcpyHostToDevice, c->stream));
  }

  // ---- dictionary: present codes in rank blocks, then the blocks' rank bases
  ALLOC(P->dict, 8 * sizeof(uint32_t) * n_dict);
  CK(cudaMemsetAsync(P->dict.p, 0, 8 * sizeof(uint32_t) * n_dict, c->stream));
  if (n_genes)
    CK(pdg::run_encode_mark(L, res_dev, gp_devp, n_genes, k, P->dict.as<uint32_t>(),
                            P->gene_genome.as<uint16_t>(), d_code_base.as<unsigned long long>(), gene_src,
                            alphabet, n_res, c->d_err, c->stream));
  const uint32_t kOrderShift = 16;  // 65536 min-hash buckets
  const uint64_t n_order_b = (uint64_t)1 << (32 - kOrderShift);
  ALLOC(tmp, pdg::scan_temp_bytes(std::max<uint64_t>(std::max<uint64_t>(n_dict, n_order_b), 24577)) + 64);
  ALLOC(d_counts, 4 * sizeof(uint32_t));  // [0] = D, [1] = max posting
  CK(cudaMemsetAsync(d_counts.p, 0, 4 * sizeof(uint32_t), c->stream));
  CK(pdg::scan_dict_blocks(L, P->dict.as<uint32_t>(), n_dict, d_counts.as<uint32_t>(), tmp.p, c->stream));
  // one synchronisation: the dictionary size, the window total, the gene
  // classes and any error found in the offsets or the letters
  unsigned long long* hb = c->h_build;
  CK(cudaMemcpyAsync(hb, d_counts.p, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(hb + 2, d_win64.as<unsigned long long>() + n_genes, sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(hb + 3, wcount64, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
  pd_status st = check_dev_err(c);  // synchronizes
  if (st != PD_OK) return st;
  const uint64_t D = (uint32_t)hb[0];
  const uint64_t W = hb[2];
  const uint32_t n_mid = (uint32_t)hb[3], n_long = (uint32_t)(hb[3] >> 32);
  const uint64_t long_total = hb[4];
  if (W > 0xFFFFFFF0ull) return fail(c, PD_ERR_ARG, "more than 2^32 k-mer windows in the dataset");
  if (!early_genomes) {
    if ((st = check_genomes()) != PD_OK) return st;
    CK(pdg::run_gene_info(L, P->genome_ptr.as<int32_t>(), n_genomes, P->La.as<uint32_t>(),
                          P->gene_genome.as<uint16_t>(), P->ginfo.as<uint32_t>(), c->stream));
  }
  P->h_genome_ptr = hgn;
  const size_t W1 = std::max<uint64_t>(W, 1);

  // ---- multiplicity vectors (and one index record per entry)
  // gene field wide enough to keep the all-ones id unused (see the packed
  // accumulator slots of k_summin.cu)
  const uint32_t gene_bits = bits_for(n_genes);
  const uint32_t cnt_bits = 32 - gene_bits;
  const uint32_t cnt_cap = std::min<uint32_t>((1u << cnt_bits) - 1u, 65535u);
  Buf mvrec;
  ALLOC(P->mv_id, sizeof(uint32_t) * W1);
  ALLOC(P->mv_cnt, sizeof(uint16_t) * W1);
  ALLOC(P->mv_n, sizeof(uint32_t) * G1);
  ALLOC(minhash, sizeof(uint32_t) * G1);
  ALLOC(mvrec, sizeof(unsigned long long) * W1);
  if (n_long) ALLOC(d_long_scratch, sizeof(unsigned long long) * long_total);
  pdg::MvOut M;
  M.mv_id = P->mv_id.as<uint32_t>();
  M.mv_cnt = P->mv_cnt.as<uint16_t>();
  M.mv_n = P->mv_n.as<uint32_t>();
  M.rec = mvrec.as<unsigned long long>();
  M.minhash = minhash.as<uint32_t>();
  M.cnt_bits = cnt_bits;
  M.cnt_cap = cnt_cap;
  M.err = c->d_err;
  M.gene_genome = P->gene_genome.as<uint16_t>();
  M.genome_code_base = d_code_base.as<unsigned long long>();
  M.gene_src = gene_src;
  M.alpha = alphabet;
  M.length_buckets = length_buckets;
  M.frozen = 0;
  if (n_genes)
    CK(pdg::run_mv_build(L, res_dev, gp_devp, P->win_off.as<uint32_t>(), n_genes, k, P->dict.as<uint32_t>(), M,
                         d_mid.as<uint32_t>(), n_mid, d_long.as<uint32_t>(), n_long,
                         d_long_scratch.as<unsigned long long>(), d_long_off.as<unsigned long long>(), c->stream));

  // ---- inverted index: stable radix sort of the index records by k-mer id
  // (records arrive in gene order, so every posting list ends up gene-sorted)
  Buf recs, rcounts, rtmp;
  ALLOC(recs, sizeof(unsigned long long) * W1);
  ALLOC(rcounts, sizeof(uint32_t) * pdg::radix_counts_words(W));
  ALLOC(rtmp, pdg::scan_temp_bytes(pdg::radix_counts_words(W)) + 64);
  ALLOC(P->post_ptr, sizeof(uint32_t) * (D + 1));
  ALLOC(P->post, sizeof(uint32_t) * W1);
  CK(cudaMemsetAsync(P->post_ptr.p, 0, sizeof(uint32_t) * (D + 1), c->stream));
  if (W && D)
    CK(pdg::run_index_sort(L, mvrec.as<unsigned long long>(), recs.as<unsigned long long>(), W, bits_for((uint32_t)D),
                           rcounts.as<uint32_t>(), rtmp.p, D, P->post.as<uint32_t>(), P->post_ptr.as<uint32_t>(),
                           c->stream));
  ALLOC(P->mv_post, sizeof(uint32_t) * W1);
  ALLOC(P->mv_plen, sizeof(uint32_t) * W1);
  if (n_genes && D)
    CK(pdg::run_mv_post(L, P->win_off.as<uint32_t>(), P->mv_n.as<uint32_t>(), P->mv_id.as<uint32_t>(), n_genes,
                        P->post_ptr.as<uint32_t>(), P->mv_post.as<uint32_t>(), P->mv_plen.as<uint32_t>(),
                        d_counts.as<uint32_t>() + 1, (unsigned long long*)(d_counts.as<uint32_t>() + 2),
                        c->stream));

  // ---- all-pairs query order: min-hash buckets
  Buf ocount;
  ALLOC(P->order, sizeof(uint32_t) * G1);
  ALLOC(ocount, sizeof(uint32_t) * (2 * n_order_b + 1));
  CK(cudaMemsetAsync(ocount.p, 0, sizeof(uint32_t) * n_order_b, c->stream));
  if (n_genes)
    CK(pdg::run_order(L, minhash.as<uint32_t>(), n_genes, kOrderShift, ocount.as<uint32_t>(),
                      P->order.as<uint32_t>(), tmp.p, c->stream));

  uint32_t* hb32 = (uint32_t*)c->h_build;  // [0] = E, [2..5] = d_counts
  CK(cudaMemcpyAsync(hb32, P->post_ptr.as<uint32_t>() + D, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(hb32 + 2, d_counts.p, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
  st = check_dev_err(c);  // synchronizes; temporaries are released after this
  if (st != PD_OK) return st;
  const uint64_t E = hb32[0];
  const uint32_t max_posting = hb32[3];
  const uint64_t n_join = ((const unsigned long long*)c->h_build)[2];  // d_counts words 2-3

  pdg::ProfilesView& v = P->view;
  v.k = k;
  v.n_genes = n_genes;
  v.n_genomes = n_genomes;
  v.n_windows = W;
  v.n_distinct = D;
  v.n_entries = E;
  v.cnt_bits = cnt_bits;
  v.cnt_cap = cnt_cap;
  v.max_posting = max_posting;
  v.n_join = n_join;
  v.win_off = P->win_off.as<uint32_t>();
  v.mv_n = P->mv_n.as<uint32_t>();
  v.mv_id = P->mv_id.as<uint32_t>();
  v.mv_cnt = P->mv_cnt.as<uint16_t>();
  v.mv_post = P->mv_post.as<uint32_t>();
  v.mv_plen = P->mv_plen.as<uint32_t>();
  v.La = P->La.as<uint32_t>();
  v.gene_genome = P->gene_genome.as<uint16_t>();
  v.ginfo = P->ginfo.as<uint32_t>();
  v.genome_ptr = P->genome_ptr.as<int32_t>();
  v.dict = P->dict.as<uint32_t>();
  v.n_dict_blocks = n_dict;
  v.post_ptr = P->post_ptr.as<uint32_t>();
  v.post = P->post.as<uint32_t>();
  v.order = P->order.as<uint32_t>();
  pd_profiles_info& in = P->info;
  in.k = k;
  in.n_genes = n_genes;
  in.n_genomes = n_genomes;
  in.n_windows = W;
  in.n_distinct = D;
  in.n_entries = E;
  in.max_posting = max_posting;
  in.n_join = n_join;
  in.count_bits = cnt_bits;
  in.alphabet = alphabet;
  in.device_bytes = P->genome_ptr.n + P->La.n + P->win_off.n + P->mv_n.n + P->mv_id.n + P->mv_cnt.n +
                    P->mv_post.n + P->mv_plen.n + P->gene_genome.n + P->ginfo.n + P->dict.n +
                    P->post_ptr.n + P->post.n + P->order.n;
  *out = guard.release();
  return PD_OK;
}

PD_API pd_status pd_build_profiles(pd_ctx* c, const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr,
                                   uint32_t n_genes, const int32_t* genome_ptr, uint32_t n_genomes, int k,
                                   pd_profiles** out) {
  if (!c || !out) return PD_ERR_ARG;
  *out = nullptr;
  try {
    return build_profiles_impl(c, residues, n_res, gene_ptr, n_genes, genome_ptr, n_genomes, k, nullptr, out);
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_build_profiles");
  }
}

PD_API pd_status pd_build_profiles_alphabet(pd_ctx* c, const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr,
                                            uint32_t n_genes, const int32_t* genome_ptr, uint32_t n_genomes,
                                            int alphabet, int k, pd_profiles** out) {
  if (!c || !out) return PD_ERR_ARG;
  *out = nullptr;
  try {
    return build_profiles_impl(c, residues, n_res, gene_ptr, n_genes, genome_ptr, n_genomes, k, nullptr, out,
                               nullptr, alphabet);
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_build_profiles_alphabet");
  }
}

PD_API pd_status pd_build_profiles_segmented(pd_ctx* c, const uint8_t* residues, uint64_t n_res,
                                             const int64_t* gene_ptr, uint32_t n_genes, const int32_t* genome_ptr,
                                             uint32_t n_genomes, const uint32_t* genome_seg, int k,
                                             pd_profiles** out) {
  if (!c || !out) return PD_ERR_ARG;
  *out = nullptr;
  if (!genome_seg) return fail(c, PD_ERR_ARG, "null genome_seg");
  if (is_device_ptr(genome_seg)) return fail(c, PD_ERR_ARG, "genome_seg must be a host array");
  try {
    return build_profiles_impl(c, residues, n_res, gene_ptr, n_genes, genome_ptr, n_genomes, k, genome_seg, out);
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_build_profiles_segmented");
  }
}

PD_API pd_status pd_profiles_get_info(const pd_profiles* P, pd_profiles_info* info) {
  if (!P || !info) return PD_ERR_ARG;
  *info = P->info;
  return PD_OK;
}

PD_API pd_status pd_profiles_genome_ptr(const pd_profiles* P, int32_t* genome_ptr) {
  if (!P || !genome_ptr) return PD_ERR_ARG;
  for (uint32_t g = 0; g <= P->info.n_genomes; ++g) genome_ptr[g] = pdg::profiles_genome_start(P, g);
  return PD_OK;
}

PD_API void pd_profiles_free(pd_profiles* P) { delete P; }


namespace {
__global__ void k_u32_to_i64(const uint32_t* __restrict__ a, uint64_t n, int64_t* __restrict__ out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = (int64_t)a[i];
}
__global__ void k_row_ids(uint32_t n_rows, const unsigned long long* __restrict__ row_ptr, int32_t* __restrict__ out) {
  for (uint32_t x = blockIdx.x; x < n_rows; x += gridDim.x)
    for (unsigned long long e = row_ptr[x] + threadIdx.x; e < row_ptr[x + 1]; e += blockDim.x) out[e] = (int32_t)x;
}
}  // namespace

PD_API pd_status pd_profiles_copy_mv(pd_ctx* c, const pd_profiles* P, int64_t* mv_ptr, uint64_t* codes,
                                     uint32_t* counts, uint32_t* La) {
  if (!c || !P) return PD_ERR_ARG;
  try {
    CK(cudaSetDevice(c->device));
    const pdg::ProfilesView& v = P->view;
    pdg::Launcher* L = &c->L;
    Buf ptr, tmp, code_of_id, d_codes, d_counts, pad_off, pad;
    ALLOC(ptr, sizeof(unsigned long long) * (v.n_genes + 1));
    ALLOC(tmp, pdg::scan_temp_bytes(v.n_genes + 1) + 64);
    CK(pdg::scan_u32_to_u64(L, v.mv_n, v.n_genes, ptr.as<unsigned long long>(), tmp.p, c->stream));
    if ((codes || counts) && v.n_genes) {
      // per-gene power-of-two scratch for the sort by code
      std::vector<uint32_t> n(v.n_genes);
      CK(cudaMemcpyAsync(n.data(), v.mv_n, sizeof(uint32_t) * v.n_genes, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      std::vector<unsigned long long> off(v.n_genes + 1, 0);
      for (uint32_t g = 0; g < v.n_genes; ++g) off[g + 1] = off[g] + (n[g] ? pdg::next_pow2(n[g]) : 0);
      ALLOC(pad_off, sizeof(unsigned long long) * (v.n_genes + 1));
      ALLOC(pad, sizeof(unsigned long long) * std::max<unsigned long long>(off[v.n_genes], 1));
      CK(cudaMemcpyAsync(pad_off.p, off.data(), sizeof(unsigned long long) * (v.n_genes + 1), cudaMemcpyHostToDevice,
                         c->stream));
      ALLOC(code_of_id, sizeof(unsigned long long) * std::max<uint64_t>(v.n_distinct, 1));
      CK(pdg::run_select_codes(L, v.dict, v.n_dict_blocks, code_of_id.as<unsigned long long>(), c->stream));
      ALLOC(d_codes, sizeof(unsigned long long) * std::max<uint64_t>(v.n_entries, 1));
      ALLOC(d_counts, sizeof(uint32_t) * std::max<uint64_t>(v.n_entries, 1));
      CK(pdg::run_export_mv(L, v, ptr.as<unsigned long long>(), pad_off.as<unsigned long long>(),
                            pad.as<unsigned long long>(), code_of_id.as<unsigned long long>(),
                            d_codes.as<unsigned long long>(), d_counts.as<uint32_t>(), c->stream));
      CK(cudaStreamSynchronize(c->stream));  // host offsets must outlive the copy
    }
    pd_status st;
    if ((st = copy_out(c, mv_ptr, ptr.p, sizeof(int64_t) * (v.n_genes + 1))) != PD_OK) return st;
    if ((st = copy_out(c, codes, d_codes.p, sizeof(uint64_t) * v.n_entries)) != PD_OK) return st;
    if ((st = copy_out(c, counts, d_counts.p, sizeof(uint32_t) * v.n_entries)) != PD_OK) return st;
    if ((st = copy_out(c, La, v.La, sizeof(uint32_t) * v.n_genes)) != PD_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    return PD_OK;
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_profiles_copy_mv");
  }
}

PD_API pd_status pd_profiles_copy_index(pd_ctx* c, const pd_profiles* P, int64_t* post_ptr, uint64_t* codes,
                                        int32_t* genes, uint32_t* counts) {
  if (!c || !P) return PD_ERR_ARG;
  try {
    CK(cudaSetDevice(c->device));
    const pdg::ProfilesView& v = P->view;
    pdg::Launcher* L = &c->L;
    Buf ptr64, code_of_id, d_genes, d_counts;
    pd_status st;
    if (post_ptr) {
      ALLOC(ptr64, sizeof(int64_t) * (v.n_distinct + 1));
      const unsigned grid = (unsigned)std::min<uint64_t>((v.n_distinct + 256) / 256 + 1, 152u * 16u);
      CK(pdg::launch_begin(L, "u32_to_i64"));
      k_u32_to_i64<<<grid, 256, 0, c->stream>>>(v.post_ptr, v.n_distinct + 1, ptr64.as<int64_t>());
      CK(pdg::launch_end(L, "u32_to_i64"));
    }
    if (codes) {
      ALLOC(code_of_id, sizeof(unsigned long long) * std::max<uint64_t>(v.n_distinct, 1));
      CK(pdg::run_select_codes(L, v.dict, v.n_dict_blocks, code_of_id.as<unsigned long long>(), c->stream));
    }
    if (genes) ALLOC(d_genes, sizeof(int32_t) * std::max<uint64_t>(v.n_entries, 1));
    if (counts) ALLOC(d_counts, sizeof(uint32_t) * std::max<uint64_t>(v.n_entries, 1));
    if ((genes || counts) && v.n_entries)
      CK(pdg::run_export_index(L, v, d_genes.as<int32_t>(), d_counts.as<uint32_t>(), c->stream));
    if ((st = copy_out(c, post_ptr, ptr64.p, sizeof(int64_t) * (v.n_distinct + 1))) != PD_OK) return st;
    if ((st = copy_out(c, codes, code_of_id.p, sizeof(uint64_t) * v.n_distinct)) != PD_OK) return st;
    if ((st = copy_out(c, genes, d_genes.p, sizeof(int32_t) * v.n_entries)) != PD_OK) return st;
    if ((st = copy_out(c, counts, d_counts.p, sizeof(uint32_t) * v.n_entries)) != PD_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    return PD_OK;
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_profiles_copy_index");
  }
}

// ------------------------------------------------------------------ sum-min + Best Hits
// Runs the shared-memory tiers, then (only if needed) the global-memory tier
// for the queries they deferred, growing the output until every row fits.
static pd_status run_hits_on(pd_ctx* c, const pdg::ProfilesView& v, const pdg::QuerySet& Q, bool emit_all,
                             pd_hits* H, uint32_t genomes_per_query);

pd_status pdh::run_hits(pd_ctx* c, const pd_profiles* P, const pdg::QuerySet& Q, bool emit_all, pd_hits* H,
                        uint32_t genomes_per_query) {
  return run_hits_on(c, P->view, Q, emit_all, H, genomes_per_query);
}

pd_status pdh::run_hits_view(pd_ctx* c, const pdg::ProfilesView& v, const pdg::QuerySet& Q, pd_hits* H,
                             uint32_t genomes_per_query) {
  return run_hits_on(c, v, Q, false, H, genomes_per_query);
}

static pd_status run_hits_on(pd_ctx* c, const pdg::ProfilesView& v, const pdg::QuerySet& Q, bool emit_all,
                             pd_hits* H, uint32_t genomes_per_query) {
  pdg::Launcher* L = &c->L;
  const uint32_t nq = Q.n_queries;
  // rows: the dataset's genes (all-pairs), or one per query (pair form, external queries)
  const uint32_t n_rows = (Q.all_pairs && !Q.q_genome) ? v.n_genes : nq;
  uint64_t cap;
  if (Q.all_pairs)
    cap = (uint64_t)nq * std::max<uint32_t>(genomes_per_query ? genomes_per_query : v.n_genomes - 1, 1) * 3 / 2 +
          4096;
  else
    cap = (uint64_t)nq * 4 + 4096;
  if (emit_all) cap = (uint64_t)nq * 64 + 4096;
  Buf counters, def1, def2;
  ALLOC(counters, 4 * sizeof(unsigned long long));
  ALLOC(H->row_off, sizeof(unsigned long long) * std::max<uint32_t>(n_rows, 1));
  ALLOC(H->row_len, sizeof(uint32_t) * std::max<uint32_t>(n_rows, 1));
  ALLOC(def1, sizeof(uint32_t) * std::max<uint32_t>(nq, 1));
  ALLOC(def2, sizeof(uint32_t) * std::max<uint32_t>(nq, 1));
  for (int attempt = 0; attempt < 3; ++attempt) {
    ALLOC(H->out_b, sizeof(uint32_t) * cap);
    ALLOC(H->out_s, sizeof(uint32_t) * cap);
    CK(cudaMemsetAsync(counters.p, 0, 4 * sizeof(unsigned long long), c->stream));
    CK(cudaMemsetAsync(H->row_len.p, 0, sizeof(uint32_t) * std::max<uint32_t>(n_rows, 1), c->stream));
    if (Q.symbest) {  // a rerun starts the reverse maxima and their tie list afresh
      CK(cudaMemsetAsync(Q.symbest, 0, sizeof(unsigned long long) * v.n_genes * v.n_genomes, c->stream));
      CK(cudaMemsetAsync(Q.tie_count, 0, sizeof(unsigned long long), c->stream));
    }
    unsigned long long* cnt = counters.as<unsigned long long>();
    pdg::HitsOut O;
    O.out_b = H->out_b.as<uint32_t>();
    O.out_s = H->out_s.as<uint32_t>();
    O.out_cap = cap;
    O.cursor = cnt + 0;
    O.walked = cnt + 1;
    O.n_def1 = (uint32_t*)(cnt + 2);
    O.n_def2 = (uint32_t*)(cnt + 3);
    O.row_off = H->row_off.as<unsigned long long>();
    O.row_len = H->row_len.as<uint32_t>();
    O.def1 = def1.as<uint32_t>();
    O.def2 = def2.as<uint32_t>();
    pdg::QuerySet Qw = Q;  // the context's walk unless the call chose one
    if (Qw.walk == PD_WALK_AUTO) Qw.walk = c->walk;
    CK(pdg::run_summin_tiers(L, v, Qw, O, c->d_err, emit_all, c->stream));
    unsigned long long h[4];
    CK(cudaMemcpyAsync(h, counters.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    pd_status st = check_dev_err(c);
    if (st != PD_OK) return st;
    const uint32_t n_def1 = (uint32_t)h[2], n_def2 = (uint32_t)h[3];
    if (n_def2 > 0) {
      pdg::BigScratch B;
      const uint32_t targets = std::max<uint32_t>(v.n_genes, 2);
      B.cap = std::max<uint32_t>(pdg::next_pow2(4 * targets), 256);  // load <= 1/4: short probe chains
      B.out_cap = pdg::next_pow2(targets);
      const uint32_t n_ctas = std::min<uint32_t>(n_def2, 64);
      Buf bk, bv, bu, bo, bpa, bpb;
      ALLOC(bk, sizeof(uint32_t) * (size_t)B.cap * n_ctas);
      ALLOC(bv, sizeof(uint32_t) * (size_t)B.cap * n_ctas);
      if (Q.filter) {
        ALLOC(bpa, sizeof(uint32_t) * (size_t)B.cap * n_ctas);
        ALLOC(bpb, sizeof(uint32_t) * (size_t)B.cap * n_ctas);
        B.vpa = bpa.as<uint32_t>();
        B.vpb = bpb.as<uint32_t>();
      }
      ALLOC(bu, sizeof(uint32_t) * (size_t)B.cap * n_ctas);
      ALLOC(bo, sizeof(unsigned long long) * (size_t)B.out_cap * n_ctas);
      B.keys = bk.as<uint32_t>();
      B.vals = bv.as<uint32_t>();
      B.used = bu.as<uint32_t>();
      B.out = bo.as<unsigned long long>();
      CK(pdg::run_summin_global(L, v, Q, O, B, n_ctas, c->d_err, emit_all, c->stream));
      CK(cudaMemcpyAsync(h, counters.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
      st = check_dev_err(c);  // synchronizes (scratch lifetime)
      if (st != PD_OK) return st;
    }
    if (h[0] <= cap) {
      H->n_hits = h[0];
      H->walked = h[1];
      H->n_deferred = n_def1;
      H->n_rows = n_rows;
      return PD_OK;
    }
    cap = h[0] + 4096;  // output did not fit: rerun with the exact size
  }
  return fail(c, PD_ERR_INTERNAL, "Best Hit output did not converge");
}

pdg::ProfilesView pdh::external_view(const pd_profiles* P, const QueryProfiles& Qp) {
  pdg::ProfilesView v = P->view;
  v.q_win_off = Qp.win_off.as<uint32_t>();
  v.q_mv_n = Qp.mv_n.as<uint32_t>();
  v.q_mv_id = Qp.mv_id.as<uint32_t>();
  v.q_mv_cnt = Qp.mv_cnt.as<uint16_t>();
  v.q_mv_post = Qp.mv_post.as<uint32_t>();
  v.q_mv_plen = Qp.mv_plen.as<uint32_t>();
  v.q_La = Qp.La.as<uint32_t>();
  return v;
}

pd_status pdh::query_profiles_impl(pd_ctx* c, const pd_profiles* P, const uint8_t* residues_dev,
                                   const int64_t* gene_ptr, uint32_t n_genes, QueryProfiles* Qp) {
  const pdg::ProfilesView& v = P->view;
  const int k = v.k;
  pdg::Launcher* L = &c->L;
  std::vector<uint32_t> La(n_genes), win_off(n_genes + 1);
  std::vector<uint32_t> mid, lng;
  std::vector<unsigned long long> lng_off;
  uint64_t W = 0, lng_total = 0;
  for (uint32_t g = 0; g < n_genes; ++g) {
    const int64_t len = gene_ptr[g + 1] - gene_ptr[g];
    if (len < 0) return fail(c, PD_ERR_ARG, "gene_ptr is decreasing");
    const uint64_t w = len >= k ? (uint64_t)(len - k + 1) : 0;
    if (w > PD_MAX_WINDOWS) return fail(c, PD_ERR_GENE_TOO_LONG, "a query gene has too many windows");
    La[g] = (uint32_t)w;
    win_off[g] = (uint32_t)W;
    W += w;
    if (W > 0xFFFFFFF0ull) return fail(c, PD_ERR_ARG, "more than 2^32 query windows");
    const uint32_t cap = pdg::mv_build_table_cap((uint32_t)w);
    if (cap > 16384) {
      lng.push_back(g);
      lng_off.push_back(lng_total);
      lng_total += cap;
    } else if (cap > 2048) {
      mid.push_back(g);
    }
  }
  win_off[n_genes] = (uint32_t)W;
  const size_t G1 = std::max<uint32_t>(n_genes, 1), W1 = std::max<uint64_t>(W, 1);
  Qp->n_genes = n_genes;
  Buf d_gp, d_mid, d_long, d_long_off, d_long_scratch, dummy;
  ALLOC(d_gp, sizeof(int64_t) * (n_genes + 1));
  ALLOC(Qp->win_off, sizeof(uint32_t) * (n_genes + 1));
  ALLOC(Qp->La, sizeof(uint32_t) * G1);
  ALLOC(Qp->mv_n, sizeof(uint32_t) * G1);
  ALLOC(Qp->mv_id, sizeof(uint32_t) * W1);
  ALLOC(Qp->mv_cnt, sizeof(uint16_t) * W1);
  ALLOC(Qp->mv_post, sizeof(uint32_t) * W1);
  ALLOC(Qp->mv_plen, sizeof(uint32_t) * W1);
  ALLOC(dummy, 16);
  CK(cudaMemcpyAsync(d_gp.p, gene_ptr, sizeof(int64_t) * (n_genes + 1), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(Qp->win_off.p, win_off.data(), sizeof(uint32_t) * (n_genes + 1), cudaMemcpyHostToDevice,
                     c->stream));
  if (n_genes) CK(cudaMemcpyAsync(Qp->La.p, La.data(), sizeof(uint32_t) * n_genes, cudaMemcpyHostToDevice, c->stream));
  if (!mid.empty()) {
    ALLOC(d_mid, sizeof(uint32_t) * mid.size());
    CK(cudaMemcpyAsync(d_mid.p, mid.data(), sizeof(uint32_t) * mid.size(), cudaMemcpyHostToDevice, c->stream));
  }
  if (!lng.empty()) {
    ALLOC(d_long, sizeof(uint32_t) * lng.size());
    ALLOC(d_long_off, sizeof(unsigned long long) * lng_off.size());
    ALLOC(d_long_scratch, sizeof(unsigned long long) * lng_total);
    CK(cudaMemcpyAsync(d_long.p, lng.data(), sizeof(uint32_t) * lng.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(d_long_off.p, lng_off.data(), sizeof(unsigned long long) * lng_off.size(),
                       cudaMemcpyHostToDevice, c->stream));
  }
  pdg::MvOut M{};
  M.mv_id = Qp->mv_id.as<uint32_t>();
  M.mv_cnt = Qp->mv_cnt.as<uint16_t>();
  M.mv_n = Qp->mv_n.as<uint32_t>();
  M.rec = nullptr;
  M.minhash = nullptr;
  M.cnt_bits = v.cnt_bits;
  M.cnt_cap = v.cnt_cap;
  M.err = c->d_err;
  M.gene_genome = nullptr;
  M.genome_code_base = nullptr;
  M.gene_src = nullptr;
  M.alpha = P->info.alphabet;
  M.length_buckets = 0;
  M.frozen = 1;
  if (n_genes) {
    CK(pdg::run_mv_build(L, residues_dev, d_gp.as<int64_t>(), Qp->win_off.as<uint32_t>(), n_genes, k, v.dict, M,
                         d_mid.as<uint32_t>(), (uint32_t)mid.size(), d_long.as<uint32_t>(),
                         (uint32_t)lng.size(), d_long_scratch.as<unsigned long long>(),
                         d_long_off.as<unsigned long long>(), c->stream));
    CK(pdg::run_mv_post(L, Qp->win_off.as<uint32_t>(), Qp->mv_n.as<uint32_t>(), Qp->mv_id.as<uint32_t>(), n_genes,
                        v.post_ptr, Qp->mv_post.as<uint32_t>(), Qp->mv_plen.as<uint32_t>(), dummy.as<uint32_t>(),
                        nullptr, c->stream));
  }
  return check_dev_err(c);  // synchronizes: the host offsets and temporaries end here
}

static pd_status hits_pair_impl(pd_ctx* c, const pd_profiles* P, uint32_t gi, uint32_t gj, bool both, bool emit_all,
                                pd_hits* H) {
  const auto& gp = P->h_genome_ptr;
  if (gi >= P->view.n_genomes || gj >= P->view.n_genomes || gi == gj)
    return fail(c, PD_ERR_ARG, "genome indices must be distinct and < n_genomes");
  pdg::QuerySet Q{};
  Q.all_pairs = 0;
  Q.qa0 = (uint32_t)gp[gi];
  Q.nA = (uint32_t)(gp[gi + 1] - gp[gi]);
  Q.ta0 = (uint32_t)gp[gj];
  Q.ta1 = (uint32_t)gp[gj + 1];
  Q.qb0 = (uint32_t)gp[gj];
  Q.tb0 = (uint32_t)gp[gi];
  Q.tb1 = (uint32_t)gp[gi + 1];
  Q.n_queries = Q.nA + (both ? (uint32_t)(gp[gj + 1] - gp[gj]) : 0u);
  H->ctx = c;
  H->all_pairs = 0;
  H->row_base = Q.qa0;
  H->col_base = Q.ta0;
  H->nA = Q.nA;
  H->qa0 = Q.qa0;
  H->qb0 = Q.qb0;
  return run_hits(c, P, Q, emit_all, H);
}

// Largest reverse-maximum table (genes x genomes x 8 B) of the symmetric form.
constexpr unsigned long long kSymMaxBytes = 4ull << 30;

// The symmetric all-pairs form (k_sym.cu): each unordered genome pair is
// walked from one side; the launch emits the forward Best Hits and keeps the
// reverse maxima, and the rows are assembled from both.
static pd_status sym_hits_impl(pd_ctx* c, const pd_profiles* P, pd_hits* H) {
  const pdg::ProfilesView& v = P->view;
  pdg::Launcher* L = &c->L;
  const uint32_t G = v.n_genes, NG = v.n_genomes;
  const unsigned long long sym_bytes = 8ull * G * NG;
  unsigned long long tie_cap = std::max<unsigned long long>(G, 1ull << 16);
  Buf symbest, ties, tcount;
  ALLOC(symbest, sym_bytes);
  ALLOC(tcount, sizeof(unsigned long long));
  for (int attempt = 0; attempt < 3; ++attempt) {
    ALLOC(ties, 2 * sizeof(unsigned long long) * tie_cap);
    pdg::QuerySet Q{};  // run_hits clears the maxima and the tie count before each launch
    Q.all_pairs = 1;
    // queries in gene order, i.e. genome by genome: the reverse maxima of the
    // query genome in flight (its slice of the genome-major array) stay in L2
    Q.order = nullptr;
    Q.q0 = 0;
    Q.n_queries = G;
    Q.symbest = symbest.as<unsigned long long>();
    Q.tie_rec = ties.as<unsigned long long>();
    Q.tie_count = tcount.as<unsigned long long>();
    Q.tie_cap = tie_cap;
    pd_hits F;
    F.ctx = c;
    F.all_pairs = 1;
    pd_status st = run_hits(c, P, Q, false, &F);  // forward rows (genomes after each query's own)
    if (st != PD_OK) return st;
    unsigned long long n_ties = 0;
    CK(cudaMemcpyAsync(&n_ties, tcount.p, sizeof(n_ties), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (n_ties > tie_cap) {  // more exact ties than the list held: run again with room for all
      tie_cap = n_ties + 4096;
      continue;
    }
    // a query handed to the next tier after its Best Hit passes records its
    // ties twice: a set keeps the first record of each pair
    Buf tie_set;
    const unsigned long long set_slots = pdg::next_pow2((uint32_t)std::min<unsigned long long>(
        std::max<unsigned long long>(2 * n_ties, 2), 1ull << 31));
    ALLOC(tie_set, sizeof(unsigned long long) * set_slots);
    CK(cudaMemsetAsync(tie_set.p, 0xFF, sizeof(unsigned long long) * set_slots, c->stream));
    pdg::SymRows R{G, NG, v.gene_genome, v.La, symbest.as<unsigned long long>(), ties.as<unsigned long long>(),
                   n_ties, tie_set.as<unsigned long long>(), set_slots - 1, F.row_off.as<unsigned long long>(),
                   F.row_len.as<uint32_t>(), F.out_b.as<uint32_t>(), F.out_s.as<uint32_t>()};
    Buf stored, tiecnt, tie_ok, total, row_ptr, tmp, tie_fill;
    const size_t G1 = std::max<uint32_t>(G, 1);
    ALLOC(stored, sizeof(uint32_t) * G1);
    ALLOC(tiecnt, sizeof(uint32_t) * G1);
    ALLOC(tie_fill, sizeof(uint32_t) * G1);
    ALLOC(tie_ok, std::max<unsigned long long>(n_ties, 1));
    ALLOC(total, sizeof(uint32_t) * G1);
    ALLOC(row_ptr, sizeof(unsigned long long) * (G + 1));
    ALLOC(tmp, pdg::scan_temp_bytes(G + 1) + 64);
    CK(cudaMemsetAsync(tiecnt.p, 0, sizeof(uint32_t) * G1, c->stream));
    CK(cudaMemsetAsync(tie_fill.p, 0, sizeof(uint32_t) * G1, c->stream));
    CK(pdg::run_sym_count(L, R, stored.as<uint32_t>(), tiecnt.as<uint32_t>(), tie_ok.as<uint8_t>(),
                          total.as<uint32_t>(), c->stream));
    CK(pdg::scan_u32_to_u64(L, total.as<uint32_t>(), G, row_ptr.as<unsigned long long>(), tmp.p, c->stream));
    unsigned long long n = 0;
    CK(cudaMemcpyAsync(&n, row_ptr.as<unsigned long long>() + G, sizeof(n), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    ALLOC(H->out_b, sizeof(uint32_t) * std::max<unsigned long long>(n, 1));
    ALLOC(H->out_s, sizeof(uint32_t) * std::max<unsigned long long>(n, 1));
    CK(pdg::run_sym_write(L, R, stored.as<uint32_t>(), tiecnt.as<uint32_t>(), tie_ok.as<uint8_t>(),
                          row_ptr.as<unsigned long long>(), tie_fill.as<uint32_t>(), H->out_b.as<uint32_t>(),
                          H->out_s.as<uint32_t>(), c->stream));
    // BBH while the reverse maxima are at hand
    Buf flag, bcnt, bstart;
    ALLOC(flag, std::max<unsigned long long>(F.out_b.n / sizeof(uint32_t), 1));
    ALLOC(bcnt, sizeof(uint32_t) * G1);
    ALLOC(bstart, sizeof(uint32_t) * (G + 1));
    CK(pdg::run_sym_bbh_count(L, R, flag.as<uint8_t>(), bcnt.as<uint32_t>(), bstart.as<uint32_t>(), tmp.p,
                              c->stream));
    uint32_t n_bbh = 0;
    CK(cudaMemcpyAsync(&n_bbh, bstart.as<uint32_t>() + G, sizeof(n_bbh), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    ALLOC(H->bbh_a, sizeof(int32_t) * std::max<uint32_t>(n_bbh, 1));
    ALLOC(H->bbh_b, sizeof(int32_t) * std::max<uint32_t>(n_bbh, 1));
    if (n_bbh)
      CK(pdg::run_sym_bbh_write(L, R, flag.as<uint8_t>(), bstart.as<uint32_t>(), H->bbh_a.as<int32_t>(),
                                H->bbh_b.as<int32_t>(), c->stream));
    st = check_dev_err(c);  // synchronizes: the forward rows and the tables end here
    if (st != PD_OK) return st;
    H->has_bbh = true;
    H->csr = true;
    H->n_bbh = n_bbh;
    H->row_off = std::move(row_ptr);
    H->row_len = std::move(total);
    H->n_rows = G;
    H->n_hits = n;
    H->walked = F.walked;
    H->n_deferred = F.n_deferred;
    return PD_OK;
  }
  return fail(c, PD_ERR_INTERNAL, "symmetric Best Hits: the tie list did not converge");
}

PD_API pd_status pd_best_hits_all(pd_ctx* c, const pd_profiles* P, pd_hits** out) {
  PhaseRange range_("pd: best hits");
  if (!c || !P || !out) return PD_ERR_ARG;
  *out = nullptr;
  try {
    CK(cudaSetDevice(c->device));
    std::unique_ptr<pd_hits> H(new pd_hits());
    H->ctx = c;
    H->all_pairs = 1;
    const uint32_t G = P->view.n_genes, NG = P->view.n_genomes;
    if (c->symmetric && G > 0 && NG >= 2 && 8ull * G * NG <= kSymMaxBytes) {
      pd_status st = sym_hits_impl(c, P, H.get());
      if (st != PD_OK) return st;
      *out = H.release();
      return PD_OK;
    }
    pdg::QuerySet Q{};
    Q.all_pairs = 1;
    Q.order = P->view.order;
    Q.q0 = 0;
    Q.n_queries = P->view.n_genes;
    pd_status st = run_hits(c, P, Q, false, H.get());
    if (st != PD_OK) return st;
    *out = H.release();
    return PD_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_best_hits_all");
  }
}

PD_API pd_status pd_best_hits_shard(pd_ctx* c, const pd_profiles* P, uint32_t shard, uint32_t n_shards,
                                    pd_hits** out) {
  PhaseRange range_("pd: best hits (shard)");
  if (!c || !P || !out) return PD_ERR_ARG;
  *out = nullptr;
  if (n_shards == 0 || shard >= n_shards) return fail(c, PD_ERR_ARG, "shard must be < n_shards");
  try {
    CK(cudaSetDevice(c->device));
    std::unique_ptr<pd_hits> H(new pd_hits());
    H->ctx = c;
    H->all_pairs = 1;
    pdg::QuerySet Q{};
    Q.all_pairs = 1;
    Q.order = P->view.order;
    Q.q0 = 0;
    const uint32_t G = P->view.n_genes;
    Q.n_queries = G;  // every order position; the kernel skips other shards' genes
    Q.n_shards = n_shards;
    Q.shard = shard;
    pd_status st = run_hits(c, P, Q, false, H.get());
    if (st != PD_OK) return st;
    *out = H.release();
    return PD_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_best_hits_shard");
  }
}

namespace {
// Rows of imported CSR pieces: for every gene the piece whose row is
// non-empty (at most one), its offset in the concatenated hit buffer and its
// length; and the checks: offsets non-decreasing from 0 to each piece's
// count, columns inside the dataset, outside the row's own genome and
// strictly ascending inside a row (the mutual check of BBH searches rows).
__global__ void k_import_rows(const unsigned long long* __restrict__ row_ptr, uint32_t n_pieces, uint32_t n_rows,
                              const unsigned long long* __restrict__ piece_n,
                              const unsigned long long* __restrict__ piece_base, const uint32_t* __restrict__ cols,
                              const uint16_t* __restrict__ gene_genome, unsigned long long* __restrict__ row_off,
                              uint32_t* __restrict__ row_len, pdg::DevErr* err) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rows; r += gridDim.x * blockDim.x) {
    unsigned long long off = 0;
    uint32_t len = 0, owners = 0;
    for (uint32_t p = 0; p < n_pieces; ++p) {
      const unsigned long long* rp = row_ptr + (size_t)p * (n_rows + 1);
      const unsigned long long b = rp[r], e = rp[r + 1];
      if (b > e || e > piece_n[p] || (r == 0 && b != 0) || (r == n_rows - 1 && e != piece_n[p])) {
        pdg::raise_error(err, PD_ERR_ARG, r);
        owners = 2;
        break;
      }
      if (e > b) {
        ++owners;
        off = piece_base[p] + b;
        len = (uint32_t)(e - b);
      }
    }
    if (owners > 1) {
      pdg::raise_error(err, PD_ERR_ARG, r);  // a row in two pieces
      len = 0;
    }
    row_off[r] = off;
    row_len[r] = len;
    uint32_t prev = 0;
    for (uint32_t x = 0; x < len; ++x) {
      const uint32_t col = cols[off + x];
      if (col >= n_rows || gene_genome[col] == gene_genome[r] || (x > 0 && col <= prev)) {
        pdg::raise_error(err, PD_ERR_ARG, r);
        break;
      }
      prev = col;
    }
  }
}
}  // namespace

PD_API pd_status pd_hits_import(pd_ctx* c, const pd_profiles* P, uint32_t n_pieces, const int64_t* const* row_ptr,
                                const int32_t* const* cols, const uint32_t* const* s, const uint64_t* n_hits,
                                pd_hits** out) {
  if (!c || !P || !out || n_pieces == 0 || !row_ptr || !cols || !s || !n_hits) return PD_ERR_ARG;
  *out = nullptr;
  try {
    CK(cudaSetDevice(c->device));
    const uint32_t G = P->view.n_genes;
    std::vector<unsigned long long> base(n_pieces), cnt(n_pieces);
    unsigned long long total = 0;
    for (uint32_t p = 0; p < n_pieces; ++p) {
      if (!row_ptr[p] || (n_hits[p] && (!cols[p] || !s[p]))) return fail(c, PD_ERR_ARG, "null piece pointer");
      base[p] = total;
      cnt[p] = n_hits[p];
      total += n_hits[p];
    }
    std::unique_ptr<pd_hits> H(new pd_hits());
    H->ctx = c;
    H->all_pairs = 1;
    H->n_rows = G;
    H->n_hits = total;
    Buf d_rp, d_meta;
    ALLOC(d_rp, sizeof(int64_t) * (size_t)(G + 1) * n_pieces);
    ALLOC(d_meta, sizeof(unsigned long long) * 2 * n_pieces);
    ALLOC(H->row_off, sizeof(unsigned long long) * std::max<uint32_t>(G, 1));
    ALLOC(H->row_len, sizeof(uint32_t) * std::max<uint32_t>(G, 1));
    ALLOC(H->out_b, sizeof(uint32_t) * std::max<unsigned long long>(total, 1));
    ALLOC(H->out_s, sizeof(uint32_t) * std::max<unsigned long long>(total, 1));
    std::vector<unsigned long long> meta(cnt);
    meta.insert(meta.end(), base.begin(), base.end());
    CK(cudaMemcpyAsync(d_meta.p, meta.data(), sizeof(unsigned long long) * 2 * n_pieces, cudaMemcpyHostToDevice,
                       c->stream));
    for (uint32_t p = 0; p < n_pieces; ++p) {
      CK(cudaMemcpyAsync(d_rp.as<int64_t>() + (size_t)p * (G + 1), row_ptr[p], sizeof(int64_t) * (G + 1),
                         cudaMemcpyDefault, c->stream));
      if (n_hits[p]) {
        CK(cudaMemcpyAsync(H->out_b.as<uint32_t>() + base[p], cols[p], sizeof(int32_t) * n_hits[p],
                           cudaMemcpyDefault, c->stream));
        CK(cudaMemcpyAsync(H->out_s.as<uint32_t>() + base[p], s[p], sizeof(uint32_t) * n_hits[p],
                           cudaMemcpyDefault, c->stream));
      }
    }
    if (G) {
      const unsigned grid = (unsigned)std::min<uint64_t>((G + 255) / 256, 152u * 8u);
      CK(pdg::launch_begin(&c->L, "import_rows"));
      k_import_rows<<<grid, 256, 0, c->stream>>>(d_rp.as<unsigned long long>(), n_pieces, G,
                                                 d_meta.as<unsigned long long>(),
                                                 d_meta.as<unsigned long long>() + n_pieces, H->out_b.as<uint32_t>(),
                                                 P->view.gene_genome, H->row_off.as<unsigned long long>(),
                                                 H->row_len.as<uint32_t>(), c->d_err);
      CK(pdg::launch_end(&c->L, "import_rows"));
    }
    pd_status st = check_dev_err(c);  // synchronizes: the staging buffers end here
    if (st != PD_OK)
      return fail(c, st, "pd_hits_import: malformed pieces (offsets, a row in two pieces, columns out of range, "
                         "in the row's own genome, or not ascending)");
    *out = H.release();
    return PD_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_hits_import");
  }
}

PD_API pd_status pd_best_hits(pd_ctx* c, const pd_profiles* P, uint32_t gi, uint32_t gj, pd_hits** out) {
  PhaseRange range_("pd: best hits (pair)");
  if (!c || !P || !out) return PD_ERR_ARG;
  *out = nullptr;
  try {
    CK(cudaSetDevice(c->device));
    std::unique_ptr<pd_hits> H(new pd_hits());
    pd_status st = hits_pair_impl(c, P, gi, gj, false, false, H.get());
    if (st != PD_OK) return st;
    *out = H.release();
    return PD_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_best_hits");
  }
}

PD_API pd_status pd_hits_get_info(const pd_hits* H, pd_hits_info* info) {
  if (!H || !info) return PD_ERR_ARG;
  info->n_rows = H->all_pairs ? H->n_rows : H->nA;
  info->n_hits = H->n_hits;
  info->row_base = H->all_pairs ? 0 : H->row_base;
  info->col_base = H->all_pairs ? 0 : H->col_base;
  info->n_deferred = H->n_deferred;
  info->postings_walked = H->walked;
  return PD_OK;
}

// CSR of the first n_rows rows of H into device buffers.
static pd_status hits_to_csr(pd_ctx* c, const pd_hits* H, uint32_t n_rows, uint32_t col_base, Buf& row_ptr,
                             Buf& cols, Buf& s, uint64_t* n_out) {
  pdg::Launcher* L = &c->L;
  Buf tmp;
  ALLOC(row_ptr, sizeof(unsigned long long) * (n_rows + 1));
  ALLOC(tmp, pdg::scan_temp_bytes(n_rows + 1) + 64);
  CK(pdg::scan_u32_to_u64(L, H->row_len.as<uint32_t>(), n_rows, row_ptr.as<unsigned long long>(), tmp.p,
                          c->stream));
  unsigned long long n = 0;
  CK(cudaMemcpyAsync(&n, row_ptr.as<unsigned long long>() + n_rows, sizeof(n), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  ALLOC(cols, sizeof(int32_t) * std::max<uint64_t>(n, 1));
  ALLOC(s, sizeof(uint32_t) * std::max<uint64_t>(n, 1));
  if (n_rows)
    CK(pdg::run_gather_rows(L, n_rows, H->row_off.as<unsigned long long>(), H->row_len.as<uint32_t>(),
                            row_ptr.as<unsigned long long>(), H->out_b.as<uint32_t>(), H->out_s.as<uint32_t>(),
                            col_base, cols.as<int32_t>(), s.as<uint32_t>(), c->stream));
  *n_out = n;
  return PD_OK;
}

PD_API pd_status pd_hits_copy(pd_ctx* c, const pd_hits* H, int64_t* row_ptr, int32_t* cols, uint32_t* s,
                              uint64_t* n_hits) {
  if (!c || !H) return PD_ERR_ARG;
  try {
    CK(cudaSetDevice(c->device));
    const uint32_t n_rows = H->all_pairs ? H->n_rows : H->nA;
    if (H->csr) {  // rows assembled in order already: copy them as they are
      pd_status st = PD_OK;
      if (n_hits) *n_hits = H->n_hits;
      if ((st = copy_out(c, row_ptr, H->row_off.p, sizeof(int64_t) * (n_rows + 1))) != PD_OK) return st;
      if ((st = copy_out(c, cols, H->out_b.p, sizeof(int32_t) * H->n_hits)) != PD_OK) return st;
      if ((st = copy_out(c, s, H->out_s.p, sizeof(uint32_t) * H->n_hits)) != PD_OK) return st;
      CK(cudaStreamSynchronize(c->stream));
      return PD_OK;
    }
    Buf rp, cb, sb;
    uint64_t n = 0;
    pd_status st = hits_to_csr(c, H, n_rows, H->all_pairs ? 0 : H->col_base, rp, cb, sb, &n);
    if (st != PD_OK) return st;
    if (n_hits) *n_hits = n;
    if ((st = copy_out(c, row_ptr, rp.p, sizeof(int64_t) * (n_rows + 1))) != PD_OK) return st;
    if ((st = copy_out(c, cols, cb.p, sizeof(int32_t) * n)) != PD_OK) return st;
    if ((st = copy_out(c, s, sb.p, sizeof(uint32_t) * n)) != PD_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    return PD_OK;
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_hits_copy");
  }
}

PD_API void pd_hits_free(pd_hits* H) { delete H; }

// ------------------------------------------------------------------ BBH
pd_status pdh::bbh_impl(pd_ctx* c, const pdg::BbhRows& R, uint64_t n_hit_slots, uint32_t a_base, uint32_t b_base,
                          pd_bbh_set* S) {
  pdg::Launcher* L = &c->L;
  Buf flags, row_cnt, row_start, tmp;
  ALLOC(flags, std::max<uint64_t>(n_hit_slots, 1));
  ALLOC(row_cnt, sizeof(uint32_t) * std::max<uint32_t>(R.n_rows, 1));
  ALLOC(row_start, sizeof(uint32_t) * (R.n_rows + 1));
  ALLOC(tmp, pdg::scan_temp_bytes(R.n_rows + 1) + 64);
  if (R.n_rows) CK(pdg::run_bbh_count(L, R, flags.as<uint8_t>(), row_cnt.as<uint32_t>(), c->stream));
  CK(pdg::scan_u32(L, row_cnt.as<uint32_t>(), R.n_rows, row_start.as<uint32_t>(), tmp.p, c->stream));
  uint32_t n = 0;
  CK(cudaMemcpyAsync(&n, row_start.as<uint32_t>() + R.n_rows, sizeof(n), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  S->ctx = c;
  S->n = n;
  ALLOC(S->a, sizeof(int32_t) * std::max<uint32_t>(n, 1));
  ALLOC(S->b, sizeof(int32_t) * std::max<uint32_t>(n, 1));
  if (R.n_rows && n)
    CK(pdg::run_bbh_write(L, R, flags.as<uint8_t>(), row_start.as<uint32_t>(), a_base, b_base, S->a.as<int32_t>(),
                          S->b.as<int32_t>(), c->stream));
  CK(cudaStreamSynchronize(c->stream));  // scratch lifetime
  return PD_OK;
}

PD_API pd_status pd_bbh_all(pd_ctx* c, const pd_profiles* P, const pd_hits* H, pd_bbh_set** out) {
  PhaseRange range_("pd: bbh");
  if (!c || !P || !H || !out) return PD_ERR_ARG;
  *out = nullptr;
  if (!H->all_pairs || H->paralog) return fail(c, PD_ERR_ARG, "pd_bbh_all needs the result of pd_best_hits_all");
  try {
    CK(cudaSetDevice(c->device));
    if (H->has_bbh) {  // found with the rows (the symmetric form)
      std::unique_ptr<pd_bbh_set> S(new pd_bbh_set());
      S->ctx = c;
      S->n = H->n_bbh;
      ALLOC(S->a, sizeof(int32_t) * std::max<uint64_t>(H->n_bbh, 1));
      ALLOC(S->b, sizeof(int32_t) * std::max<uint64_t>(H->n_bbh, 1));
      if (H->n_bbh) {
        CK(cudaMemcpyAsync(S->a.p, H->bbh_a.p, sizeof(int32_t) * H->n_bbh, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(S->b.p, H->bbh_b.p, sizeof(int32_t) * H->n_bbh, cudaMemcpyDeviceToDevice, c->stream));
      }
      CK(cudaStreamSynchronize(c->stream));
      *out = S.release();
      return PD_OK;
    }
    pdg::BbhRows R{};
    R.all_pairs = 1;
    R.n_rows = H->n_rows;
    R.gene_genome = P->view.gene_genome;
    R.genome_ptr = P->view.genome_ptr;
    R.row_off = H->row_off.as<unsigned long long>();
    R.row_len = H->row_len.as<uint32_t>();
    R.hit_b = H->out_b.as<uint32_t>();
    std::unique_ptr<pd_bbh_set> S(new pd_bbh_set());
    pd_status st = bbh_impl(c, R, H->out_b.n / sizeof(uint32_t), 0, 0, S.get());
    if (st != PD_OK) return st;
    *out = S.release();
    return PD_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_bbh_all");
  }
}

static pd_status set_filter(pd_ctx* c, const pd_filter* f, pdg::QuerySet* Q) {
  if (!f) return fail(c, PD_ERR_ARG, "null filter");
  if (f->theta_den == 0 || f->tau_den == 0 || f->theta_num > f->theta_den || f->tau_num > f->tau_den)
    return fail(c, PD_ERR_ARG, "theta and tau must be fractions in [0, 1] with a denominator >= 1");
  Q->filter = 1;
  Q->theta_num = f->theta_num;
  Q->theta_den = f->theta_den;
  Q->tau_num = f->tau_num;
  Q->tau_den = f->tau_den;
  return PD_OK;
}

PD_API pd_status pd_best_hits_all_filtered(pd_ctx* c, const pd_profiles* P, const pd_filter* f, pd_hits** out) {
  if (!c || !P || !out) return PD_ERR_ARG;
  *out = nullptr;
  try {
    CK(cudaSetDevice(c->device));
    std::unique_ptr<pd_hits> H(new pd_hits());
    H->ctx = c;
    H->all_pairs = 1;
    pdg::QuerySet Q{};
    Q.all_pairs = 1;
    Q.order = P->view.order;
    Q.n_queries = P->view.n_genes;
    pd_status st = set_filter(c, f, &Q);
    if (st != PD_OK) return st;
    if ((st = run_hits(c, P, Q, false, H.get())) != PD_OK) return st;
    *out = H.release();
    return PD_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_best_hits_all_filtered");
  }
}

PD_API pd_status pd_best_hits_filtered(pd_ctx* c, const pd_profiles* P, uint32_t gi, uint32_t gj, const pd_filter* f,
                                       pd_hits** out) {
  if (!c || !P || !out) return PD_ERR_ARG;
  *out = nullptr;
  try {
    CK(cudaSetDevice(c->device));
    const auto& gp = P->h_genome_ptr;
    if (gi >= P->view.n_genomes || gj >= P->view.n_genomes || gi == gj)
      return fail(c, PD_ERR_ARG, "genome indices must be distinct and < n_genomes");
    std::unique_ptr<pd_hits> H(new pd_hits());
    pdg::QuerySet Q{};
    pd_status st = set_filter(c, f, &Q);
    if (st != PD_OK) return st;
    Q.all_pairs = 0;
    Q.qa0 = (uint32_t)gp[gi];
    Q.nA = (uint32_t)(gp[gi + 1] - gp[gi]);
    Q.ta0 = (uint32_t)gp[gj];
    Q.ta1 = (uint32_t)gp[gj + 1];
    Q.n_queries = Q.nA;
    H->ctx = c;
    H->all_pairs = 0;
    H->row_base = Q.qa0;
    H->col_base = Q.ta0;
    H->nA = Q.nA;
    H->qa0 = Q.qa0;
    if ((st = run_hits(c, P, Q, false, H.get())) != PD_OK) return st;
    *out = H.release();
    return PD_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_best_hits_filtered");
  }
}

PD_API pd_status pd_paralog_hits(pd_ctx* c, const pd_profiles* P, pd_hits** out) {
  if (!c || !P || !out) return PD_ERR_ARG;
  *out = nullptr;
  try {
    CK(cudaSetDevice(c->device));
    std::unique_ptr<pd_hits> H(new pd_hits());
    H->ctx = c;
    pdg::QuerySet Q{};
    Q.all_pairs = 0;
    Q.paralog = 1;
    Q.q0 = 0;
    Q.n_queries = P->view.n_genes;
    pd_status st = run_hits(c, P, Q, false, H.get());
    if (st != PD_OK) return st;
    H->all_pairs = 1;  // rows are all genes, columns global ids
    H->paralog = 1;
    H->n_rows = P->view.n_genes;
    *out = H.release();
    return PD_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_paralog_hits");
  }
}

PD_API pd_status pd_paralog_bbh(pd_ctx* c, const pd_profiles* P, const pd_hits* H, pd_bbh_set** out) {
  if (!c || !P || !H || !out) return PD_ERR_ARG;
  *out = nullptr;
  if (!H->paralog) return fail(c, PD_ERR_ARG, "pd_paralog_bbh needs the result of pd_paralog_hits");
  try {
    CK(cudaSetDevice(c->device));
    pdg::BbhRows R{};
    R.all_pairs = 1;
    R.paralog = 1;
    R.n_rows = H->n_rows;
    R.gene_genome = P->view.gene_genome;
    R.genome_ptr = P->view.genome_ptr;
    R.row_off = H->row_off.as<unsigned long long>();
    R.row_len = H->row_len.as<uint32_t>();
    R.hit_b = H->out_b.as<uint32_t>();
    std::unique_ptr<pd_bbh_set> S(new pd_bbh_set());
    pd_status st = bbh_impl(c, R, H->out_b.n / sizeof(uint32_t), 0, 0, S.get());
    if (st != PD_OK) return st;
    *out = S.release();
    return PD_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_paralog_bbh");
  }
}

PD_API pd_status pd_bbh(pd_ctx* c, const pd_profiles* P, uint32_t gi, uint32_t gj, pd_bbh_set** out) {
  PhaseRange range_("pd: bbh (pair)");
  if (!c || !P || !out) return PD_ERR_ARG;
  *out = nullptr;
  try {
    CK(cudaSetDevice(c->device));
    pd_hits H;
    pd_status st = hits_pair_impl(c, P, gi, gj, true, false, &H);
    if (st != PD_OK) return st;
    pdg::BbhRows R{};
    R.all_pairs = 0;
    R.n_rows = H.n_rows;
    R.nA = H.nA;
    R.qa0 = H.qa0;
    R.qb0 = H.qb0;
    R.row_off = H.row_off.as<unsigned long long>();
    R.row_len = H.row_len.as<uint32_t>();
    R.hit_b = H.out_b.as<uint32_t>();
    std::unique_ptr<pd_bbh_set> S(new pd_bbh_set());
    st = bbh_impl(c, R, H.out_b.n / sizeof(uint32_t), H.qa0, H.qb0, S.get());
    if (st != PD_OK) return st;
    *out = S.release();
    return PD_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_bbh");
  }
}

PD_API pd_status pd_bbh_copy(pd_ctx* c, const pd_bbh_set* S, int32_t* a, int32_t* b, uint64_t* n_pairs) {
  if (!c || !S) return PD_ERR_ARG;
  try {
    if (n_pairs) *n_pairs = S->n;
    pd_status st;
    if ((st = copy_out(c, a, S->a.p, sizeof(int32_t) * S->n)) != PD_OK) return st;
    if ((st = copy_out(c, b, S->b.p, sizeof(int32_t) * S->n)) != PD_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    return PD_OK;
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_bbh_copy");
  }
}

PD_API uint64_t pd_bbh_count(const pd_bbh_set* S) { return S ? S->n : 0; }

PD_API void pd_bbh_free(pd_bbh_set* S) { delete S; }

// ------------------------------------------------------------------ sum-min pairs
PD_API pd_status pd_summin_pairs(pd_ctx* c, const pd_profiles* P, uint32_t gi, uint32_t gj, int32_t* a, int32_t* b,
                                 uint32_t* s, uint64_t* n) {
  if (!c || !P) return PD_ERR_ARG;
  try {
    CK(cudaSetDevice(c->device));
    pd_hits H;
    pd_status st = hits_pair_impl(c, P, gi, gj, false, true, &H);
    if (st != PD_OK) return st;
    Buf rp, cb, sb;
    uint64_t total = 0;
    st = hits_to_csr(c, &H, H.nA, H.col_base, rp, cb, sb, &total);
    if (st != PD_OK) return st;
    if (!a) {
      if (n) *n = total;
      return PD_OK;
    }
    if (n && *n < total) return fail(c, PD_ERR_ARG, "output holds fewer entries than pd_summin_pairs produces");
    if (n) *n = total;
    Buf ra;
    ALLOC(ra, sizeof(int32_t) * std::max<uint64_t>(total, 1));
    if (H.nA) {
      CK(pdg::launch_begin(&c->L, "row_ids"));
      k_row_ids<<<std::min<uint32_t>(H.nA, 152u * 8u), 128, 0, c->stream>>>(H.nA, rp.as<unsigned long long>(),
                                                                            ra.as<int32_t>());
      CK(pdg::launch_end(&c->L, "row_ids"));
    }
    if ((st = copy_out(c, a, ra.p, sizeof(int32_t) * total)) != PD_OK) return st;
    if ((st = copy_out(c, b, cb.p, sizeof(int32_t) * total)) != PD_OK) return st;
    if ((st = copy_out(c, s, sb.p, sizeof(uint32_t) * total)) != PD_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    return PD_OK;
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_summin_pairs");
  }
}
