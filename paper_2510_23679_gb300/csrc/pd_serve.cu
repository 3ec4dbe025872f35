// pd_serve.cu -- served form: a pangenome index resident on the device and a
// request loop that compares incoming genomes with it (pd_index_* in pd.h).
//
// Each incoming genome X asks for Best Hits BH(a, G_j) of its genes a in every
// resident genome G_j (Eq. (8)) and for its Bidirectional Best Hits with the
// resident genes (Eq. (9)); X then becomes resident itself.
//
// Request loop (one worker thread, one stream, one memory pool):
//   * submit copies the genome to the host queue and stamps it with the
//     resident set it will be compared with (its snapshot: the genomes
//     resident at submission);
//   * the resident genomes are indexed in two levels: a base index and a
//     delta index of the genomes inserted since the base was built.  After
//     each tick the delta is rebuilt over the new residents, or, once its
//     windows pass a quarter of the base's, everything is merged into a new
//     base -- so a tick never rebuilds the whole resident set;
//   * continuous batching: whenever the GPU is free the worker admits queued
//     requests in arrival order while the HBM estimate of the tick stays within
//     the budget, and runs them together: per level, the tick's genes are
//     profiled against the level's dictionary (k-mers the level does not hold
//     are left out of the walk but count in La) and ONE sum-min / Best Hit
//     launch sequence answers every gene of every admitted genome against it;
//   * each query is limited to the genes of its snapshot, so a result does not
//     depend on which other requests shared its tick;
//   * every resident genome lies in exactly one level, so the Best Hits of a
//     row are the union of the levels' rows (base genes first);
//   * the reverse direction of Eq. (9) -- is a among the Best Hits of b in X?
//     -- needs, for every resident gene b, its best ratio over the genes of X.
//     The sum-min kernel keeps that maximum per (b, X) in global memory while
//     it selects the forward Best Hits; a pair (a, b) is a BBH when b is a
//     forward Best Hit of a and the ratio of (a, b) equals b's maximum over X.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "pd.h"
#include "pd_host.cuh"
#include "pd_internal.cuh"

using namespace pdh;

struct pd_reply {
  pd_reply_info info{};
  std::string err;
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> cols;
  std::vector<uint32_t> s;
  std::vector<int32_t> bbh_a, bbh_b;
};

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t ticket = 0;
  std::vector<uint8_t> res;
  std::vector<int64_t> gene_ptr;  // local CSR, n_genes + 1 entries
  uint32_t snapshot = 0;          // resident genomes this request is compared with
  uint64_t windows = 0;
  int64_t t_submit = 0;
};

// Device bytes of one tick beyond the resident data: the profile build over
// W windows and G genes, the Best Hit output and the reverse-maximum table.
uint64_t tick_bytes(uint64_t W, uint64_t G, uint64_t tick_genes, uint64_t res_genes, uint64_t res_genomes,
                    uint64_t tick_genomes) {
  return 48 * W + 64 * G + 8 * res_genes * tick_genomes + 24 * tick_genes * (res_genomes + 1) + (64ull << 20);
}

// Mutual check of the served Best Hits: warp per row of the tick.
__global__ void k_serve_bbh_count(uint32_t n_rows, const unsigned long long* __restrict__ row_ptr,
                                  const int32_t* __restrict__ cols, const uint32_t* __restrict__ s,
                                  const uint32_t* __restrict__ La_q, const uint32_t* __restrict__ La_t,
                                  const uint32_t* __restrict__ q_genome, uint32_t stride,
                                  const unsigned long long* __restrict__ colbest, uint8_t* __restrict__ flag,
                                  uint32_t* __restrict__ cnt) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rows; r += warps) {
    const uint32_t x = q_genome[r];
    const unsigned long long lo = row_ptr[r], hi = row_ptr[r + 1];
    uint32_t n = 0;
    for (unsigned long long i = lo + lane; i < hi; i += 32) {
      const uint32_t b = (uint32_t)cols[i], sv = s[i];
      const unsigned long long cb = colbest[(size_t)b * stride + x];
      const bool f = pdg::ratio_equal(sv, La_q[r] + La_t[b] - sv, (uint32_t)(cb >> 32), (uint32_t)cb);
      flag[i] = f ? 1 : 0;
      n += f ? 1u : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (lane == 0) cnt[r] = n;
  }
}

__global__ void k_serve_bbh_write(uint32_t n_rows, const unsigned long long* __restrict__ row_ptr,
                                  const int32_t* __restrict__ cols, const uint8_t* __restrict__ flag,
                                  const uint32_t* __restrict__ start, int32_t* __restrict__ out_a,
                                  int32_t* __restrict__ out_b) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rows; r += warps) {
    const unsigned long long lo = row_ptr[r], hi = row_ptr[r + 1];
    uint32_t pos = start[r];
    for (unsigned long long i0 = lo; i0 < hi; i0 += 32) {
      const unsigned long long i = i0 + lane;
      const bool f = i < hi && flag[i];
      const uint32_t m = __ballot_sync(0xffffffffu, f);
      if (f) {
        const uint32_t p = pos + __popc(m & ((1u << lane) - 1u));
        out_a[p] = (int32_t)r;
        out_b[p] = cols[i];
      }
      pos += __popc(m);
    }
  }
}

__global__ void k_iota(uint32_t* out, uint32_t n, uint32_t base) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = base + i;
}

unsigned grid_of(uint64_t items, unsigned per_block, unsigned cap) {
  uint64_t b = (items + per_block - 1) / per_block;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, cap));
}

#define PD_KLAUNCH(name, ...)               \
  do {                                      \
    CK(pdg::launch_begin(&c->L, name));     \
    __VA_ARGS__;                            \
    CK(pdg::launch_end(&c->L, name));       \
  } while (0)

uint64_t windows_of(const std::vector<int64_t>& gp, size_t g0, size_t g1, int k) {
  uint64_t w = 0;
  for (size_t g = g0; g < g1; ++g) {
    const int64_t len = gp[g + 1] - gp[g];
    if (len >= k) w += (uint64_t)(len - k + 1);
  }
  return w;
}

}  // namespace

// One level of the resident index: the profiles of resident genomes
// [genome0, genome1) (genes [gene0, gene1), global numbering).
struct Level {
  std::unique_ptr<pd_profiles> P;
  uint32_t genome0 = 0, genome1 = 0, gene0 = 0, gene1 = 0;
  uint64_t windows = 0;
  bool empty() const { return !P || gene1 == gene0; }
  uint64_t bytes() const { return P ? P->info.device_bytes : 0; }
};

struct pd_index {
  pd_ctx* c = nullptr;  // worker context: own stream and memory pool
  cudaStream_t stream = nullptr;
  int device = 0, k = 0;
  uint64_t budget = 0;
  uint32_t max_tick = 64;
  // resident data (owned by the worker once it runs)
  Buf res;
  uint64_t res_used = 0;
  std::vector<int64_t> gene_ptr;
  std::vector<int32_t> genome_ptr;
  std::vector<uint64_t> genome_windows;  // windows of each resident genome at k
  Level base, delta;
  // shared with the API threads
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::map<uint64_t, std::unique_ptr<pd_reply>> done;
  uint64_t next_ticket = 1;
  uint32_t committed = 0;
  uint64_t committed_windows = 0;
  uint64_t committed_genes = 0;
  uint64_t committed_res = 0;  // resident residues (res_used as of the last commit)
  std::vector<int32_t> committed_genome_ptr;
  uint64_t resident_bytes = 0;
  bool stop = false;
  bool hold = false;  // admission paused: queued requests wait (pd_index_hold)
  // The levels index genomes [0, covered); genomes committed since then make
  // them stale.  A request is answered from levels covering its snapshot.
  uint32_t covered = 0;
  bool stale = false;
  std::thread worker;
  pd_index_info stats{};
  // Background merge: a builder thread with a context (stream, memory pool)
  // of its own builds the next base from a copy of the residues while the
  // worker keeps answering ticks from the current base and delta.
  pd_ctx* bc = nullptr;
  cudaStream_t bstream = nullptr;
  std::thread builder;
  std::mutex bmu;
  bool merging = false;     // a builder thread was started and not yet joined
  bool merge_done = false;  // the builder finished (its status in merge_status)
  pd_status merge_status = PD_OK;
  Level merged;             // its result: the profiles of genomes [0, merged.genome1)
  Buf merge_res;            // the builder's copy of the residues (its context)
  uint64_t merge_bytes = 0; // device bytes the builder holds or will hold

  ~pd_index() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv_work.notify_all();
    if (worker.joinable()) worker.join();
    if (builder.joinable()) builder.join();
    if (c) {
      cudaSetDevice(device);
      base.P.reset();
      delta.P.reset();
      merged.P.reset();
      merge_res.release();
      res.release();
      cudaStreamSynchronize(stream);
      if (bstream) cudaStreamSynchronize(bstream);
      pd_ctx_destroy(c);
      if (bc) pd_ctx_destroy(bc);
    }
    if (stream) cudaStreamDestroy(stream);
    if (bstream) cudaStreamDestroy(bstream);
  }
};

namespace {

// Profiles of resident genomes [g0, g1) as one level, built on context c
// from residues `res` (device) and the host offsets gene_ptr / genome_ptr.
pd_status build_level_on(pd_ctx* c, int k, const uint8_t* res, const std::vector<int64_t>& gene_ptr,
                         const std::vector<int32_t>& genome_ptr, const std::vector<uint64_t>& genome_windows,
                         uint32_t g0, uint32_t g1, Level* L) {
  L->P.reset();
  L->genome0 = g0;
  L->genome1 = g1;
  L->gene0 = (uint32_t)genome_ptr[g0];
  L->gene1 = (uint32_t)genome_ptr[g1];
  L->windows = 0;
  for (uint32_t i = g0; i < g1; ++i) L->windows += genome_windows[i];
  if (g1 == g0 || L->gene1 == L->gene0) return PD_OK;
  const int64_t r0 = gene_ptr[L->gene0];
  std::vector<int64_t> gp(gene_ptr.begin() + L->gene0, gene_ptr.begin() + L->gene1 + 1);
  for (auto& x : gp) x -= r0;
  std::vector<int32_t> gn(genome_ptr.begin() + g0, genome_ptr.begin() + g1 + 1);
  for (auto& x : gn) x -= (int32_t)L->gene0;
  pd_profiles* P = nullptr;
  pd_status st = build_profiles_impl(c, res + r0, (uint64_t)gp.back(), gp.data(), L->gene1 - L->gene0, gn.data(),
                                     g1 - g0, k, nullptr, &P);
  if (st != PD_OK) return st;
  L->P.reset(P);
  return PD_OK;
}

pd_status build_level(pd_index* I, uint32_t g0, uint32_t g1, Level* L) {
  return build_level_on(I->c, I->k, I->res.as<uint8_t>(), I->gene_ptr, I->genome_ptr, I->genome_windows, g0, g1, L);
}

// Builder thread: the profiles of genomes [0, n) from the snapshot taken by
// start_merge (host offsets passed by value, residues in merge_res).
void builder_main(pd_index* I, uint32_t n, std::vector<int64_t> gene_ptr, std::vector<int32_t> genome_ptr,
                  std::vector<uint64_t> genome_windows) {
  cudaSetDevice(I->device);
  Level L;
  pd_status st;
  try {
    st = build_level_on(I->bc, I->k, I->merge_res.as<uint8_t>(), gene_ptr, genome_ptr, genome_windows, 0, n, &L);
    if (st == PD_OK && cudaStreamSynchronize(I->bstream) != cudaSuccess) st = PD_ERR_CUDA;
  } catch (...) {
    st = PD_ERR_INTERNAL;
  }
  std::lock_guard<std::mutex> lk(I->bmu);
  I->merged = std::move(L);
  I->merge_status = st;
  I->merge_done = true;
}

// Starts a background merge of the committed genomes [0, n) (the worker's
// thread, between ticks): the builder gets a copy of the residues -- the
// worker may grow (move) its own buffer meanwhile -- and of the host offsets.
pd_status start_merge(pd_index* I, uint32_t n) {
  pd_ctx* c = I->c;
  if (!I->bc) {
    // the background merge yields the SMs to ticks: lowest stream priority
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CK(cudaStreamCreateWithPriority(&I->bstream, cudaStreamNonBlocking, least));
    pd_status st = pd_ctx_create(I->device, I->bstream, nullptr, nullptr, nullptr, &I->bc);
    if (st != PD_OK) return fail(c, st, "could not create the builder context");
    uint64_t keep = I->budget;
    CK(cudaMemPoolSetAttribute(I->bc->pool, cudaMemPoolAttrReleaseThreshold, &keep));
  }
  const uint64_t r_end = (uint64_t)I->gene_ptr[I->genome_ptr[n]];
  if (!I->merge_res.alloc(I->bc, std::max<uint64_t>(r_end, 1)))
    return fail(c, PD_ERR_OOM, "residue copy for the background merge");
  // the residues were written on the worker's stream; the copy reads them on
  // the builder's and ends before the worker can move its buffer
  cudaEvent_t ev;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(I->bstream, ev, 0);
  if (e == cudaSuccess && r_end) e = cudaMemcpyAsync(I->merge_res.p, I->res.p, r_end, cudaMemcpyDeviceToDevice, I->bstream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(I->bstream);
  cudaEventDestroy(ev);
  if (e != cudaSuccess) return fail_cuda(c, e, "residue copy for the background merge");
  I->merging = true;
  I->merge_done = false;
  I->merge_bytes = I->merge_res.n + I->base.bytes() + I->delta.bytes();  // the new base is about their size
  std::vector<int64_t> gp(I->gene_ptr.begin(), I->gene_ptr.begin() + I->genome_ptr[n] + 1);
  std::vector<int32_t> gn(I->genome_ptr.begin(), I->genome_ptr.begin() + n + 1);
  std::vector<uint64_t> gw(I->genome_windows.begin(), I->genome_windows.begin() + n);
  I->builder = std::thread(builder_main, I, n, std::move(gp), std::move(gn), std::move(gw));
  return PD_OK;
}

// Brings the levels up to the committed genomes (the worker's thread, between
// ticks).  The delta is rebuilt over the genomes after the base.  Once it holds
// more than a quarter of the base's windows, a builder thread merges
// everything into a new base in the background while ticks go on against the
// old base and the delta; when it is done the new base replaces the old one
// and the delta shrinks to the genomes committed since the merge began.
pd_status refresh_levels(pd_index* I) {
  const uint32_t n = (uint32_t)I->genome_ptr.size() - 1;
  // ---- a finished background merge takes over
  bool done = false;
  {
    std::lock_guard<std::mutex> lk(I->bmu);
    done = I->merging && I->merge_done;
  }
  if (done) {
    I->builder.join();
    I->merging = false;
    I->merge_res.release();  // the builder's stream is idle: its work was synchronized
    I->merge_bytes = 0;
    if (I->merge_status == PD_OK) {
      I->base = std::move(I->merged);  // the old base's last use ended with the previous tick
      I->delta = Level();
      I->delta.genome0 = I->delta.genome1 = I->base.genome1;
      I->delta.gene0 = I->delta.gene1 = I->base.gene1;
    }
    I->merged = Level();
  }
  const uint32_t nb = I->base.genome1;
  if (I->delta.genome0 == nb && I->delta.genome1 == n && (I->delta.P || nb == n)) return PD_OK;
  uint64_t dw = 0;
  for (uint32_t i = nb; i < n; ++i) dw += I->genome_windows[i];
  I->delta.P.reset();
  if (!I->merging && 4 * dw > I->base.windows) {
    pd_status st = start_merge(I, n);
    if (st != PD_OK) {  // no background merge: merge here, as the fallback
      I->base.P.reset();
      st = build_level(I, 0, n, &I->base);
      if (st != PD_OK) return st;
      I->delta = Level();
      I->delta.genome0 = I->delta.genome1 = n;
      I->delta.gene0 = I->delta.gene1 = (uint32_t)I->genome_ptr[n];
      return PD_OK;
    }
  }
  return build_level(I, nb, n, &I->delta);
}

// One level's answer for the tick's genes: rows in CSR (level-local target
// ids) and the BBH pairs (tick row, level-local target), on the host.
struct LevelAnswer {
  std::vector<unsigned long long> rp;
  std::vector<int32_t> cols, pa, pb;
  std::vector<uint32_t> s;
};

pd_status answer_level(pd_index* I, const Level& L, const uint8_t* tick_res, const std::vector<int64_t>& tick_gp,
                       const std::vector<uint32_t>& q_genome, const std::vector<uint32_t>& snap_gene_end,
                       LevelAnswer* out) {
  pd_ctx* c = I->c;
  const uint32_t n_q = (uint32_t)tick_gp.size() - 1, n_tick = (uint32_t)snap_gene_end.size();
  out->rp.assign(n_q + 1, 0);
  if (L.empty() || n_q == 0) return PD_OK;
  const uint32_t nL = L.gene1 - L.gene0;
  QueryProfiles Qp;
  pd_status st = query_profiles_impl(c, L.P.get(), tick_res, tick_gp.data(), n_q, &Qp);
  if (st != PD_OK) return st;
  const pdg::ProfilesView V = external_view(L.P.get(), Qp);
  std::vector<uint32_t> tgt_end(n_tick);
  for (uint32_t x = 0; x < n_tick; ++x)
    tgt_end[x] = snap_gene_end[x] <= L.gene0 ? 0u : std::min<uint32_t>(snap_gene_end[x], L.gene1) - L.gene0;
  Buf order, d_qg, d_tgt, colbest;
  ALLOC(order, sizeof(uint32_t) * n_q);
  ALLOC(d_qg, sizeof(uint32_t) * n_q);
  ALLOC(d_tgt, sizeof(uint32_t) * n_tick);
  ALLOC(colbest, sizeof(unsigned long long) * (size_t)nL * n_tick);
  CK(cudaMemcpyAsync(d_qg.p, q_genome.data(), sizeof(uint32_t) * n_q, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d_tgt.p, tgt_end.data(), sizeof(uint32_t) * n_tick, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(colbest.p, 0, sizeof(unsigned long long) * (size_t)nL * n_tick, c->stream));
  PD_KLAUNCH("serve_iota", (k_iota<<<grid_of(n_q, 256, 152u * 4u), 256, 0, c->stream>>>(order.as<uint32_t>(), n_q,
                                                                                         0u)));
  pdg::QuerySet Q{};
  Q.all_pairs = 1;
  Q.order = order.as<uint32_t>();
  Q.n_queries = n_q;
  Q.q_genome = d_qg.as<uint32_t>();
  Q.tgt_end = d_tgt.as<uint32_t>();
  Q.colbest = colbest.as<unsigned long long>();
  Q.col_genome0 = 0;
  Q.col_stride = n_tick;
  pd_hits H;
  H.ctx = c;
  if ((st = run_hits_view(c, V, Q, &H, std::max<uint32_t>(L.genome1 - L.genome0, 1))) != PD_OK) return st;

  Buf row_ptr, cols, sv, tmp, flag, cnt, start, pa, pb;
  ALLOC(row_ptr, sizeof(unsigned long long) * (n_q + 1));
  ALLOC(tmp, pdg::scan_temp_bytes(n_q + 1) + 64);
  CK(pdg::scan_u32_to_u64(&c->L, H.row_len.as<uint32_t>(), n_q, row_ptr.as<unsigned long long>(), tmp.p,
                          c->stream));
  unsigned long long n_hits = 0;
  CK(cudaMemcpyAsync(&n_hits, row_ptr.as<unsigned long long>() + n_q, sizeof(n_hits), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  ALLOC(cols, sizeof(int32_t) * std::max<unsigned long long>(n_hits, 1));
  ALLOC(sv, sizeof(uint32_t) * std::max<unsigned long long>(n_hits, 1));
  CK(pdg::run_gather_rows(&c->L, n_q, H.row_off.as<unsigned long long>(), H.row_len.as<uint32_t>(),
                          row_ptr.as<unsigned long long>(), H.out_b.as<uint32_t>(), H.out_s.as<uint32_t>(), 0,
                          cols.as<int32_t>(), sv.as<uint32_t>(), c->stream));
  ALLOC(flag, std::max<unsigned long long>(n_hits, 1));
  ALLOC(cnt, sizeof(uint32_t) * n_q);
  ALLOC(start, sizeof(uint32_t) * (n_q + 1));
  PD_KLAUNCH("serve_bbh_count",
             (k_serve_bbh_count<<<grid_of((uint64_t)n_q * 32, 256, 152u * 16u), 256, 0, c->stream>>>(
                 n_q, row_ptr.as<unsigned long long>(), cols.as<int32_t>(), sv.as<uint32_t>(), Qp.La.as<uint32_t>(),
                 L.P->view.La, d_qg.as<uint32_t>(), n_tick, colbest.as<unsigned long long>(), flag.as<uint8_t>(),
                 cnt.as<uint32_t>())));
  CK(pdg::scan_u32(&c->L, cnt.as<uint32_t>(), n_q, start.as<uint32_t>(), tmp.p, c->stream));
  uint32_t n_bbh = 0;
  CK(cudaMemcpyAsync(&n_bbh, start.as<uint32_t>() + n_q, sizeof(n_bbh), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  ALLOC(pa, sizeof(int32_t) * std::max<uint32_t>(n_bbh, 1));
  ALLOC(pb, sizeof(int32_t) * std::max<uint32_t>(n_bbh, 1));
  if (n_bbh)
    PD_KLAUNCH("serve_bbh_write", (k_serve_bbh_write<<<grid_of((uint64_t)n_q * 32, 256, 152u * 16u), 256, 0,
                                                       c->stream>>>(n_q, row_ptr.as<unsigned long long>(),
                                                                    cols.as<int32_t>(), flag.as<uint8_t>(),
                                                                    start.as<uint32_t>(), pa.as<int32_t>(),
                                                                    pb.as<int32_t>())));
  out->cols.resize(n_hits);
  out->s.resize(n_hits);
  out->pa.resize(n_bbh);
  out->pb.resize(n_bbh);
  CK(cudaMemcpyAsync(out->rp.data(), row_ptr.p, sizeof(unsigned long long) * (n_q + 1), cudaMemcpyDeviceToHost,
                     c->stream));
  if (n_hits) {
    CK(cudaMemcpyAsync(out->cols.data(), cols.p, sizeof(int32_t) * n_hits, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(out->s.data(), sv.p, sizeof(uint32_t) * n_hits, cudaMemcpyDeviceToHost, c->stream));
  }
  if (n_bbh) {
    CK(cudaMemcpyAsync(out->pa.data(), pa.p, sizeof(int32_t) * n_bbh, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(out->pb.data(), pb.p, sizeof(int32_t) * n_bbh, cudaMemcpyDeviceToHost, c->stream));
  }
  return check_dev_err(c);  // synchronizes
}

// Appends the genomes of `tick` to the resident data and answers every
// request of the tick against both levels (the levels hold the committed
// genomes; the tick's genomes join them when the levels are next refreshed).
pd_status run_tick(pd_index* I, std::vector<Request>& tick, std::vector<std::unique_ptr<pd_reply>>& replies) {
  PhaseRange range_("pd: served tick");
  pd_ctx* c = I->c;
  const uint32_t n_tick = (uint32_t)tick.size();
  const uint32_t g_res = (uint32_t)I->genome_ptr.size() - 1;
  if (g_res + n_tick > PD_MAX_GENOMES) return fail(c, PD_ERR_BUDGET, "the index holds at most PD_MAX_GENOMES genomes");
  uint64_t add = 0;
  for (auto& r : tick) add += r.res.size();
  // ---- residues: grow the resident buffer (doubling), then append
  if (I->res_used + add > I->res.n || !I->res.p) {
    Buf bigger;
    const uint64_t want = std::max<uint64_t>(I->res_used + add, std::max<uint64_t>(2 * I->res.n, 1 << 20));
    ALLOC(bigger, want);
    if (I->res_used) CK(cudaMemcpyAsync(bigger.p, I->res.p, I->res_used, cudaMemcpyDeviceToDevice, c->stream));
    // the levels' profiles do not point into the residues, so moving them is safe
    I->res = std::move(bigger);
  }
  const uint64_t tick_r0 = I->res_used;
  uint64_t off = tick_r0;
  std::vector<int64_t> tick_gp(1, 0);
  std::vector<uint32_t> q_genome, snap_gene_end(n_tick);
  for (uint32_t x = 0; x < n_tick; ++x) {
    const Request& r = tick[x];
    if (!r.res.empty())
      CK(cudaMemcpyAsync(I->res.as<uint8_t>() + off, r.res.data(), r.res.size(), cudaMemcpyHostToDevice, c->stream));
    for (size_t g = 1; g < r.gene_ptr.size(); ++g) {
      I->gene_ptr.push_back((int64_t)off + r.gene_ptr[g]);
      tick_gp.push_back((int64_t)(off - tick_r0) + r.gene_ptr[g]);
      q_genome.push_back(x);
    }
    I->genome_ptr.push_back((int32_t)(I->gene_ptr.size() - 1));
    I->genome_windows.push_back(r.windows);
    snap_gene_end[x] = (uint32_t)I->genome_ptr[r.snapshot];
    off += r.res.size();
  }
  I->res_used = off;

  // ---- every level answers every gene of the tick
  LevelAnswer A[2];
  const Level* levels[2] = {&I->base, &I->delta};
  for (int l = 0; l < 2; ++l) {
    pd_status st = answer_level(I, *levels[l], I->res.as<uint8_t>() + tick_r0, tick_gp, q_genome, snap_gene_end,
                                &A[l]);
    if (st != PD_OK) return st;
  }

  // ---- per request: rows = base part then delta part (global resident ids)
  uint32_t r0 = 0;
  size_t p[2] = {0, 0};
  for (uint32_t x = 0; x < n_tick; ++x) {
    const uint32_t nx = (uint32_t)tick[x].gene_ptr.size() - 1;
    std::unique_ptr<pd_reply> R(new pd_reply());
    R->row_ptr.resize(nx + 1, 0);
    for (uint32_t i = 0; i < nx; ++i) {
      const uint32_t r = r0 + i;
      for (int l = 0; l < 2; ++l) {
        if (A[l].cols.empty()) continue;
        const int32_t g0 = (int32_t)levels[l]->gene0;
        for (unsigned long long e = A[l].rp[r]; e < A[l].rp[r + 1]; ++e) {
          R->cols.push_back(A[l].cols[e] + g0);
          R->s.push_back(A[l].s[e]);
        }
      }
      R->row_ptr[i + 1] = (int64_t)R->cols.size();
      for (int l = 0; l < 2; ++l) {
        const int32_t g0 = (int32_t)levels[l]->gene0;
        while (p[l] < A[l].pa.size() && (uint32_t)A[l].pa[p[l]] == r) {
          R->bbh_a.push_back((int32_t)i);
          R->bbh_b.push_back(A[l].pb[p[l]] + g0);
          ++p[l];
        }
      }
    }
    R->info.ticket = tick[x].ticket;
    R->info.status = PD_OK;
    R->info.snapshot_genomes = tick[x].snapshot;
    R->info.n_genes = nx;
    R->info.n_hits = R->cols.size();
    R->info.n_bbh = R->bbh_a.size();
    R->info.tick_requests = n_tick;
    replies.push_back(std::move(R));
    r0 += nx;
  }
  return PD_OK;
}

void worker_main(pd_index* I) {
  cudaSetDevice(I->device);
  for (;;) {
    std::vector<Request> tick;
    bool refresh = false;
    {
      std::unique_lock<std::mutex> lk(I->mu);
      // work: queued requests (unless held), or stale levels to refresh while
      // nothing waits
      I->cv_work.wait(lk, [&] {
        return I->stop || (!I->hold && !I->queue.empty()) || (I->stale && (I->hold || I->queue.empty()));
      });
      if (I->stop) return;
      // The levels are refreshed only when a queued request needs the genomes
      // committed since (its snapshot is past the levels' coverage), or when
      // no request waits; requests queued during a tick were stamped before
      // its commit and are answered at once from the levels as they are.
      const bool needs = !I->hold && !I->queue.empty() && I->queue.front().snapshot > I->covered;
      refresh = needs || (I->stale && (I->hold || I->queue.empty()));
      // admission in arrival order while the tick's estimate fits the budget
      uint64_t W = I->committed_windows, G = I->committed_genes, tick_genes = 0;
      while (!refresh && !I->queue.empty() && tick.size() < I->max_tick) {
        const Request& r = I->queue.front();
        if (r.snapshot > I->covered) break;  // needs a refresh first
        const uint64_t ng = r.gene_ptr.size() - 1;
        const uint64_t est = I->resident_bytes + tick_bytes(W + r.windows, G + ng, tick_genes + ng,
                                                            I->committed_genes, I->committed, tick.size() + 1) +
                             2 * (I->res_used + r.res.size());
        if (est > I->budget && !tick.empty()) break;
        if (est > I->budget) {  // cannot fit even alone: answer with an error
          std::unique_ptr<pd_reply> R(new pd_reply());
          R->info.ticket = r.ticket;
          R->info.status = PD_ERR_BUDGET;
          R->info.t_submit_ns = r.t_submit;
          R->info.t_done_ns = now_ns();
          R->err = "request does not fit the HBM budget next to the resident index";
          I->done[r.ticket] = std::move(R);
          I->queue.pop_front();
          I->cv_done.notify_all();
          continue;
        }
        W += r.windows;
        G += ng;
        tick_genes += ng;
        tick.push_back(std::move(I->queue.front()));
        I->queue.pop_front();
      }
    }
    if (refresh) {
      // take the committed genomes into the levels (the delta is rebuilt, or
      // a background merge begins or is taken over)
      pd_status rs;
      try {
        rs = refresh_levels(I);
      } catch (...) {
        rs = PD_ERR_INTERNAL;
      }
      const uint32_t cov = (I->delta.P || I->delta.genome1 == I->delta.genome0)
                               ? std::max(I->base.genome1, I->delta.genome1)
                               : I->base.genome1;
      std::lock_guard<std::mutex> lk2(I->mu);
      I->covered = cov;
      // a failed idle refresh is not retried until the next commit or a
      // request that needs it (which then receives the error)
      I->stale = rs == PD_OK && cov < (uint32_t)I->genome_ptr.size() - 1;
      I->resident_bytes = I->res.n + I->base.bytes() + I->delta.bytes() + I->merge_bytes;
      if (rs != PD_OK && !I->queue.empty() && I->queue.front().snapshot > cov) {
        // the refresh failed: answer the waiting request with the error rather than retry forever
        Request r = std::move(I->queue.front());
        I->queue.pop_front();
        std::unique_ptr<pd_reply> R(new pd_reply());
        R->info.ticket = r.ticket;
        R->info.status = rs;
        R->info.t_submit_ns = r.t_submit;
        R->info.t_done_ns = now_ns();
        R->err = I->c->err;
        I->done[r.ticket] = std::move(R);
        I->cv_done.notify_all();
      }
      continue;
    }
    if (tick.empty()) continue;
    const int64_t t_start = now_ns();
    std::vector<std::unique_ptr<pd_reply>> replies;
    const uint64_t res_used0 = I->res_used;
    const size_t gp0 = I->gene_ptr.size(), gn0 = I->genome_ptr.size(), gw0 = I->genome_windows.size();
    pd_status st;
    try {
      st = run_tick(I, tick, replies);
    } catch (...) {
      st = PD_ERR_INTERNAL;
      I->c->err = "exception in the request loop";
    }
    const int64_t t_done = now_ns();
    std::unique_lock<std::mutex> lk(I->mu);
    if (st == PD_OK) {
      I->committed += (uint32_t)tick.size();
      I->committed_genes = I->gene_ptr.size() - 1;
      I->committed_res = I->res_used;
      for (auto& r : tick) I->committed_windows += r.windows;
      I->committed_genome_ptr = I->genome_ptr;
      I->stats.ticks += 1;
      I->stats.max_tick_requests = std::max<uint32_t>(I->stats.max_tick_requests, (uint32_t)tick.size());
      for (auto& R : replies) {
        R->info.t_start_ns = t_start;
        R->info.t_done_ns = t_done;
      }
      for (size_t x = 0; x < tick.size(); ++x) {
        replies[x]->info.t_submit_ns = tick[x].t_submit;
        I->done[tick[x].ticket] = std::move(replies[x]);
      }
      I->stats.requests_done += tick.size();
    } else {
      // roll the resident data back; every request of the tick gets the error
      I->res_used = res_used0;
      I->gene_ptr.resize(gp0);
      I->genome_ptr.resize(gn0);
      I->genome_windows.resize(gw0);
      for (auto& r : tick) {
        std::unique_ptr<pd_reply> R(new pd_reply());
        R->info.ticket = r.ticket;
        R->info.status = st;
        R->info.t_submit_ns = r.t_submit;
        R->info.t_start_ns = t_start;
        R->info.t_done_ns = t_done;
        R->err = I->c->err;
        I->done[r.ticket] = std::move(R);
      }
    }
    if (st == PD_OK) I->stale = true;  // the tick's genomes are resident, not yet indexed
    I->cv_done.notify_all();
  }
}

pd_status index_create(pd_ctx* caller, const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr,
                       uint32_t n_genes, const int32_t* genome_ptr, uint32_t n_genomes, int k, uint64_t hbm_budget,
                       pd_index** out) {
  pd_ctx* c = caller;
  if (k < 1 || k > PD_MAX_K) return fail(c, PD_ERR_K_RANGE, "k must be in [1, " + std::to_string(PD_MAX_K) + "]");
  if (!gene_ptr || !genome_ptr || (n_res && !residues)) return fail(c, PD_ERR_ARG, "null argument");
  if (n_genomes < 1 || n_genomes > PD_MAX_GENOMES) return fail(c, PD_ERR_ARG, "n_genomes must be in [1, 4096]");
  std::unique_ptr<pd_index> I(new pd_index());
  I->device = caller->device;
  I->k = k;
  I->budget = hbm_budget;
  CK(cudaSetDevice(I->device));
  // ticks run at the highest stream priority, ahead of a background merge
  int least = 0, greatest = 0;
  CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  CK(cudaStreamCreateWithPriority(&I->stream, cudaStreamNonBlocking, greatest));
  pd_status st = pd_ctx_create(I->device, I->stream, nullptr, nullptr, nullptr, &I->c);
  if (st != PD_OK) return fail(caller, st, "could not create the index context");
  c = I->c;
  uint64_t keep = hbm_budget;  // the index's pool keeps up to the budget for reuse
  CK(cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep));
  // resident offsets on the host
  I->gene_ptr.resize(n_genes + 1);
  I->genome_ptr.resize(n_genomes + 1);
  CK(cudaMemcpy(I->gene_ptr.data(), gene_ptr, sizeof(int64_t) * (n_genes + 1), cudaMemcpyDefault));
  CK(cudaMemcpy(I->genome_ptr.data(), genome_ptr, sizeof(int32_t) * (n_genomes + 1), cudaMemcpyDefault));
  if (I->gene_ptr[0] != 0 || (uint64_t)I->gene_ptr[n_genes] != n_res || I->genome_ptr[0] != 0 ||
      (uint32_t)I->genome_ptr[n_genomes] != n_genes)
    return fail(caller, PD_ERR_ARG, "malformed gene_ptr or genome_ptr");
  if (!I->res.alloc(c, std::max<uint64_t>(n_res, 1 << 20))) return fail(caller, PD_ERR_OOM, "resident residues");
  if (n_res) {
    if (cudaMemcpyAsync(I->res.p, residues, n_res, cudaMemcpyDefault, I->stream) != cudaSuccess)
      return fail_cuda(caller, cudaGetLastError(), "copy of the resident residues");
  }
  I->res_used = n_res;
  for (uint32_t i = 0; i < n_genomes; ++i)
    I->genome_windows.push_back(windows_of(I->gene_ptr, I->genome_ptr[i], I->genome_ptr[i + 1], k));
  st = build_level(I.get(), 0, n_genomes, &I->base);
  if (st != PD_OK) return fail(caller, st, c->err);
  I->delta.genome0 = I->delta.genome1 = n_genomes;
  I->delta.gene0 = I->delta.gene1 = n_genes;
  I->committed = n_genomes;
  I->committed_genes = n_genes;
  I->committed_windows = windows_of(I->gene_ptr, 0, n_genes, k);
  I->committed_genome_ptr = I->genome_ptr;
  I->committed_res = n_res;
  I->covered = n_genomes;
  I->resident_bytes = I->res.n + I->base.bytes();
  if (I->resident_bytes > hbm_budget) return fail(caller, PD_ERR_BUDGET, "the resident index exceeds the budget");
  I->worker = std::thread(worker_main, I.get());
  *out = I.release();
  return PD_OK;
}

}  // namespace

PD_API pd_status pd_index_create(pd_ctx* c, const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr,
                                 uint32_t n_genes, const int32_t* genome_ptr, uint32_t n_genomes, int k,
                                 uint64_t hbm_budget, pd_index** out) {
  if (!c || !out) return PD_ERR_ARG;
  *out = nullptr;
  try {
    return index_create(c, residues, n_res, gene_ptr, n_genes, genome_ptr, n_genomes, k, hbm_budget, out);
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_index_create");
  }
}

PD_API pd_status pd_index_submit(pd_index* I, const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr,
                                 uint32_t n_genes, uint64_t* ticket) {
  if (!I || !ticket || !gene_ptr || (n_res && !residues)) return PD_ERR_ARG;
  try {
    Request r;
    r.gene_ptr.assign(gene_ptr, gene_ptr + n_genes + 1);
    if (r.gene_ptr[0] != 0 || (uint64_t)r.gene_ptr[n_genes] != n_res) return PD_ERR_ARG;
    for (uint32_t g = 0; g < n_genes; ++g) {
      if (r.gene_ptr[g + 1] < r.gene_ptr[g]) return PD_ERR_ARG;
      if (r.gene_ptr[g + 1] - r.gene_ptr[g] - I->k + 1 > (int64_t)PD_MAX_WINDOWS) return PD_ERR_GENE_TOO_LONG;
    }
    // letters are checked here: the tick profiles the genome against the
    // resident dictionary, which has no place for foreign letters
    static const char kLetters[] = "ACDEFGHIKLMNPQRSTVWY";
    bool valid[256] = {false};
    for (const char* q = kLetters; *q; ++q) valid[(uint8_t)*q] = true;
    for (uint64_t i = 0; i < n_res; ++i)
      if (!valid[residues[i]]) return PD_ERR_ALPHABET;
    r.res.assign(residues, residues + n_res);
    r.windows = windows_of(r.gene_ptr, 0, n_genes, I->k);
    r.t_submit = now_ns();
    std::lock_guard<std::mutex> lk(I->mu);
    const uint64_t est = I->resident_bytes +
                         tick_bytes(I->committed_windows + r.windows, I->committed_genes + n_genes, n_genes,
                                    I->committed_genes, I->committed, 1) +
                         2 * (I->committed_res + n_res);
    if (est > I->budget) return PD_ERR_BUDGET;
    if (I->committed + I->queue.size() + 1 > PD_MAX_GENOMES) return PD_ERR_BUSY;
    r.ticket = I->next_ticket++;
    r.snapshot = I->committed;
    *ticket = r.ticket;
    I->queue.push_back(std::move(r));
    I->cv_work.notify_one();
    return PD_OK;
  } catch (const std::bad_alloc&) {
    return PD_ERR_OOM;
  } catch (...) {
    return PD_ERR_INTERNAL;
  }
}

PD_API pd_status pd_index_poll(pd_index* I, uint64_t ticket, int wait_ms, pd_reply** out) {
  if (!I || !out) return PD_ERR_ARG;
  *out = nullptr;
  std::unique_lock<std::mutex> lk(I->mu);
  if (ticket == 0 || ticket >= I->next_ticket) return PD_ERR_ARG;
  auto ready = [&] { return I->done.count(ticket) != 0; };
  if (!ready()) {
    if (wait_ms < 0)
      I->cv_done.wait(lk, ready);
    else if (!I->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready))
      return PD_ERR_TIMEOUT;
  }
  auto it = I->done.find(ticket);
  *out = it->second.release();
  I->done.erase(it);
  return PD_OK;
}

PD_API pd_status pd_index_hold(pd_index* I, int hold) {
  if (!I) return PD_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(I->mu);
    I->hold = hold != 0;
  }
  I->cv_work.notify_all();
  return PD_OK;
}

PD_API pd_status pd_index_get_info(pd_index* I, pd_index_info* info) {
  if (!I || !info) return PD_ERR_ARG;
  std::lock_guard<std::mutex> lk(I->mu);
  *info = I->stats;
  info->k = I->k;
  info->n_genomes = I->committed;
  info->n_genes = I->committed_genes;
  info->queued = (uint32_t)I->queue.size();
  info->device_bytes = I->resident_bytes;
  info->budget = I->budget;
  return PD_OK;
}

PD_API pd_status pd_index_genome_ptr(pd_index* I, uint32_t n_genomes, int32_t* genome_ptr) {
  if (!I || !genome_ptr) return PD_ERR_ARG;
  std::lock_guard<std::mutex> lk(I->mu);
  if (n_genomes > I->committed) return PD_ERR_ARG;
  std::copy(I->committed_genome_ptr.begin(), I->committed_genome_ptr.begin() + n_genomes + 1, genome_ptr);
  return PD_OK;
}

PD_API void pd_index_free(pd_index* I) { delete I; }

PD_API pd_status pd_reply_get_info(const pd_reply* R, pd_reply_info* info) {
  if (!R || !info) return PD_ERR_ARG;
  *info = R->info;
  return PD_OK;
}

PD_API const char* pd_reply_error(const pd_reply* R) { return R ? R->err.c_str() : "null reply"; }

PD_API pd_status pd_reply_copy(const pd_reply* R, int64_t* row_ptr, int32_t* cols, uint32_t* s, int32_t* bbh_a,
                               int32_t* bbh_b) {
  if (!R) return PD_ERR_ARG;
  if (R->info.status != PD_OK) return (pd_status)R->info.status;
  if (row_ptr) std::copy(R->row_ptr.begin(), R->row_ptr.end(), row_ptr);
  if (cols) std::copy(R->cols.begin(), R->cols.end(), cols);
  if (s) std::copy(R->s.begin(), R->s.end(), s);
  if (bbh_a) std::copy(R->bbh_a.begin(), R->bbh_a.end(), bbh_a);
  if (bbh_b) std::copy(R->bbh_b.begin(), R->bbh_b.end(), bbh_b);
  return PD_OK;
}

PD_API void pd_reply_free(pd_reply* R) { delete R; }
