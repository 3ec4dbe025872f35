// pd_batch.cu -- batched genome-pair jobs (pd_bbh_batch in pd.h).
//
// Many independent jobs "compare genome A with genome B at k" (Algorithms
// 2-3 per job) are served by few launch sequences instead of one per job:
//
//   1. jobs are grouped by k and cut into chunks (bounded windows, bounded
//      dictionary: codes x segments);
//   2. a chunk is ONE segmented profile build (each job its own k-mer
//      namespace, so postings of one job never reach another job's genes),
//      ONE all-pairs Best Hit pass (every gene of every job queried in the
//      same persistent sum-min launch; own-genome targets are skipped and
//      other jobs' genes can never be candidates), and ONE BBH pass;
//   3. the chunk results are scattered into job order: per-row Best Hit
//      lengths, one scan over all rows of the batch, then the rows themselves
//      with columns made local to the partner genome; BBH pairs likewise with
//      one scan over the jobs.
//
// Genes are read in place from the input residues (a per-gene source offset),
// so a chunk's genomes need not be consecutive in the input.
#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "pd.h"
#include "pd_host.cuh"
#include "pd_internal.cuh"

using namespace pdh;

struct pd_batch {
  pd_ctx* ctx = nullptr;
  pd_batch_info info{};
  Buf row_ptr, cols, s, job_ptr, a, b;
};

namespace {

constexpr uint64_t kDefaultChunkWindows = 1ull << 29;
// Dictionary codes per chunk (segments x 20^k; one bit each, 256 MiB of
// bits): small enough that its random marks mostly hit L2.
constexpr uint64_t kChunkDictCodes = 2048ull << 20;

// One job of a chunk: where its genes sit in the chunk and in the batch.
struct ChunkJob {
  uint32_t job;        // batch job index
  uint32_t a0, nA;     // chunk gene ids of genome A: a0 .. a0+nA-1
  uint32_t b0, nB;     // ... of genome B (b0 = a0 + nA)
  uint32_t bbh_lo;     // first BBH pair of the job in the chunk's pair list (device-written)
  unsigned long long row0;  // first batch row of the job
};

// Row lengths of a chunk's Best Hits into batch row order.
__global__ void k_rows_len(const ChunkJob* __restrict__ jobs, uint32_t n_jobs, const uint32_t* __restrict__ row_len,
                           uint32_t* __restrict__ batch_len) {
  for (uint32_t j = blockIdx.x; j < n_jobs; j += gridDim.x) {
    const ChunkJob J = jobs[j];
    for (uint32_t r = threadIdx.x; r < J.nA + J.nB; r += blockDim.x) batch_len[J.row0 + r] = row_len[J.a0 + r];
  }
}

// Best Hit rows of a chunk into the batch CSR, one warp per row; columns
// become indices inside the partner genome.
__global__ void k_rows_fill(const ChunkJob* __restrict__ jobs, uint32_t n_jobs,
                            const unsigned long long* __restrict__ row_off, const uint32_t* __restrict__ row_len,
                            const uint32_t* __restrict__ hit_b, const uint32_t* __restrict__ hit_s,
                            const unsigned long long* __restrict__ batch_ptr, int32_t* __restrict__ cols,
                            uint32_t* __restrict__ s) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
  for (uint32_t j = blockIdx.x; j < n_jobs; j += gridDim.x) {
    const ChunkJob J = jobs[j];
    for (uint32_t r = warp; r < J.nA + J.nB; r += n_warps) {
      const uint32_t g = J.a0 + r;
      const uint32_t partner0 = r < J.nA ? J.b0 : J.a0;
      const unsigned long long src = row_off[g], dst = batch_ptr[J.row0 + r];
      const uint32_t len = row_len[g];
      for (uint32_t i = lane; i < len; i += 32) {
        cols[dst + i] = (int32_t)(hit_b[src + i] - partner0);
        s[dst + i] = hit_s[src + i];
      }
    }
  }
}

__device__ __forceinline__ uint32_t lower_bound_i32(const int32_t* a, uint32_t n, int32_t x) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// BBH pairs of each chunk job: the chunk's pairs are sorted by a and a job's
// A genes are one range, so its pairs are the run [lower_bound(a0),
// lower_bound(a0 + nA)).
__global__ void k_bbh_runs(ChunkJob* __restrict__ jobs, uint32_t n_jobs, const int32_t* __restrict__ pa, uint32_t n_pairs,
                           uint32_t* __restrict__ job_cnt) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n_jobs; j += gridDim.x * blockDim.x) {
    const uint32_t lo = lower_bound_i32(pa, n_pairs, (int32_t)jobs[j].a0);
    const uint32_t hi = lower_bound_i32(pa, n_pairs, (int32_t)(jobs[j].a0 + jobs[j].nA));
    jobs[j].bbh_lo = lo;
    job_cnt[jobs[j].job] = hi - lo;
  }
}

__global__ void k_bbh_fill(const ChunkJob* __restrict__ jobs, uint32_t n_jobs, const int32_t* __restrict__ pa,
                           const int32_t* __restrict__ pb, const unsigned long long* __restrict__ job_ptr,
                           int32_t* __restrict__ a, int32_t* __restrict__ b) {
  for (uint32_t j = blockIdx.x; j < n_jobs; j += gridDim.x) {
    const ChunkJob J = jobs[j];
    const unsigned long long dst = job_ptr[J.job], n = job_ptr[J.job + 1] - dst;
    for (unsigned long long i = threadIdx.x; i < n; i += blockDim.x) {
      a[dst + i] = pa[J.bbh_lo + i] - (int32_t)J.a0;
      b[dst + i] = pb[J.bbh_lo + i] - (int32_t)J.b0;
    }
  }
}

unsigned grid_of(uint64_t items, unsigned per_block, unsigned cap) {
  uint64_t b = (items + per_block - 1) / per_block;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, cap));
}

#define PD_KLAUNCH(name, ...)                            \
  do {                                                   \
    CK(pdg::launch_begin(&c->L, name));                  \
    __VA_ARGS__;                                         \
    CK(pdg::launch_end(&c->L, name));                    \
  } while (0)

// Results of one chunk, kept until the batch is assembled.
struct ChunkOut {
  std::vector<ChunkJob> jobs;
  Buf d_jobs;
  pd_hits hits;
  pd_bbh_set bbh;
};

pd_status batch_impl(pd_ctx* c, const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr, uint32_t n_genes,
                     const int32_t* genome_ptr, uint32_t n_genomes, const uint32_t* jobs, const int32_t* job_k,
                     uint32_t n_jobs, const pd_batch_tuning* tuning, pd_batch** out) {
  if ((n_jobs && (!jobs || !job_k)) || !gene_ptr || !genome_ptr || (n_res && !residues))
    return fail(c, PD_ERR_ARG, "null argument");
  if (n_jobs && (is_device_ptr(jobs) || is_device_ptr(job_k)))
    return fail(c, PD_ERR_ARG, "jobs and job_k must be host arrays");
  if (n_genomes < 1) return fail(c, PD_ERR_ARG, "n_genomes must be >= 1");
  CK(cudaSetDevice(c->device));
  const uint64_t max_windows = (tuning && tuning->max_chunk_windows) ? tuning->max_chunk_windows
                                                                     : kDefaultChunkWindows;

  // ---- offsets on the host
  std::vector<int64_t> hg(n_genes + 1);
  std::vector<int32_t> hgn(n_genomes + 1);
  CK(cudaMemcpyAsync(hg.data(), gene_ptr, sizeof(int64_t) * (n_genes + 1), cudaMemcpyDefault, c->stream));
  CK(cudaMemcpyAsync(hgn.data(), genome_ptr, sizeof(int32_t) * (n_genomes + 1), cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (hg[0] != 0 || (uint64_t)hg[n_genes] != n_res) return fail(c, PD_ERR_ARG, "gene_ptr must run from 0 to n_res");
  if (hgn[0] != 0 || (uint32_t)hgn[n_genomes] != n_genes)
    return fail(c, PD_ERR_ARG, "genome_ptr must run from 0 to n_genes");
  for (uint32_t i = 0; i < n_genomes; ++i)
    if (hgn[i + 1] < hgn[i]) return fail(c, PD_ERR_ARG, "genome_ptr is decreasing at " + std::to_string(i));
  for (uint32_t g = 0; g < n_genes; ++g)
    if (hg[g + 1] < hg[g]) return fail(c, PD_ERR_ARG, "gene_ptr is decreasing at " + std::to_string(g));
  for (uint32_t j = 0; j < n_jobs; ++j) {
    if (jobs[2 * j] >= n_genomes || jobs[2 * j + 1] >= n_genomes || jobs[2 * j] == jobs[2 * j + 1])
      return fail(c, PD_ERR_ARG, "job " + std::to_string(j) + " needs two distinct genome indices < n_genomes");
    if (job_k[j] < 1 || job_k[j] > PD_MAX_K)
      return fail(c, PD_ERR_K_RANGE, "job " + std::to_string(j) + ": k must be in [1, " +
                                          std::to_string(PD_MAX_K) + "]");
  }
  auto genes_of = [&](uint32_t i) { return (uint32_t)(hgn[i + 1] - hgn[i]); };
  auto windows_of = [&](uint32_t i, int k) {
    uint64_t w = 0;
    for (int32_t g = hgn[i]; g < hgn[i + 1]; ++g) {
      const int64_t len = hg[g + 1] - hg[g];
      if (len >= k) w += (uint64_t)(len - k + 1);
    }
    return w;
  };

  // ---- residues on the device (one copy of host input)
  Buf d_all;
  const uint8_t* res_dev = residues;
  if (n_res && !is_device_ptr(residues)) {
    ALLOC(d_all, n_res);
    CK(cudaMemcpyAsync(d_all.p, residues, n_res, cudaMemcpyHostToDevice, c->stream));
    res_dev = d_all.as<uint8_t>();
  }

  // ---- batch rows
  std::unique_ptr<pd_batch> B(new pd_batch());
  B->ctx = c;
  std::vector<unsigned long long> row0(n_jobs + 1, 0);
  for (uint32_t j = 0; j < n_jobs; ++j) row0[j + 1] = row0[j] + genes_of(jobs[2 * j]) + genes_of(jobs[2 * j + 1]);
  const uint64_t n_rows = row0[n_jobs];
  Buf row_len, job_cnt, tmp;
  ALLOC(row_len, sizeof(uint32_t) * std::max<uint64_t>(n_rows, 1));
  ALLOC(job_cnt, sizeof(uint32_t) * (n_jobs + 1));
  ALLOC(B->row_ptr, sizeof(unsigned long long) * (n_rows + 1));
  ALLOC(B->job_ptr, sizeof(unsigned long long) * (n_jobs + 1));
  ALLOC(tmp, pdg::scan_temp_bytes(std::max<uint64_t>(n_rows, n_jobs) + 1) + 64);
  CK(cudaMemsetAsync(row_len.p, 0, sizeof(uint32_t) * std::max<uint64_t>(n_rows, 1), c->stream));
  CK(cudaMemsetAsync(job_cnt.p, 0, sizeof(uint32_t) * (n_jobs + 1), c->stream));

  // ---- chunks: jobs grouped by k (stable), cut by windows, dictionary and genome limits
  std::vector<uint32_t> by_k(n_jobs);
  for (uint32_t j = 0; j < n_jobs; ++j) by_k[j] = j;
  std::stable_sort(by_k.begin(), by_k.end(), [&](uint32_t x, uint32_t y) { return job_k[x] < job_k[y]; });
  std::vector<std::unique_ptr<ChunkOut>> chunks;
  uint64_t walked = 0, n_hits_total = 0;
  size_t pos = 0;
  while (pos < by_k.size()) {
    const int k = job_k[by_k[pos]];
    uint64_t n_codes = 1;
    for (int t = 0; t < k; ++t) n_codes *= 20;
    uint64_t max_jobs = std::max<uint64_t>(1, kChunkDictCodes / n_codes);
    max_jobs = std::min<uint64_t>(max_jobs, PD_MAX_GENOMES / 2);
    if (tuning && tuning->max_chunk_jobs) max_jobs = std::min<uint64_t>(max_jobs, tuning->max_chunk_jobs);
    std::vector<uint32_t> cj;  // batch jobs of this chunk
    uint64_t W = 0;
    while (pos < by_k.size() && job_k[by_k[pos]] == k && cj.size() < max_jobs) {
      const uint32_t j = by_k[pos];
      const uint64_t w = windows_of(jobs[2 * j], k) + windows_of(jobs[2 * j + 1], k);
      if (!cj.empty() && W + w > max_windows) break;
      cj.push_back(j);
      W += w;
      ++pos;
    }

    // chunk dataset: genomes A0, B0, A1, B1, ...; segment = job within the chunk
    std::unique_ptr<ChunkOut> C(new ChunkOut());
    std::vector<uint32_t> genomes;
    std::vector<uint32_t> seg;
    for (uint32_t x = 0; x < cj.size(); ++x) {
      genomes.push_back(jobs[2 * cj[x]]);
      genomes.push_back(jobs[2 * cj[x] + 1]);
      seg.push_back(x);
      seg.push_back(x);
    }
    // chunk gene lengths (CSR) and where each gene starts in the input
    std::vector<int32_t> cgn(genomes.size() + 1, 0);
    std::vector<int64_t> cg(1, 0), src;
    for (size_t i = 0; i < genomes.size(); ++i) {
      const uint32_t gi = genomes[i];
      for (int32_t g = hgn[gi]; g < hgn[gi + 1]; ++g) {
        cg.push_back(cg.back() + (hg[g + 1] - hg[g]));
        src.push_back(hg[g]);
      }
      cgn[i + 1] = cgn[i] + (int32_t)genes_of(gi);
    }
    const uint32_t chunk_genes = (uint32_t)cgn.back();
    Buf d_src;
    ALLOC(d_src, sizeof(int64_t) * std::max<size_t>(src.size(), 1));
    if (!src.empty())
      CK(cudaMemcpyAsync(d_src.p, src.data(), sizeof(int64_t) * src.size(), cudaMemcpyHostToDevice, c->stream));
    pd_profiles* Praw = nullptr;
    const int length_buckets = (tuning && tuning->query_order == 1) ? 0 : 1;
    pd_status st = build_profiles_impl(c, res_dev, (uint64_t)cg.back(), cg.data(), chunk_genes, cgn.data(),
                                       (uint32_t)genomes.size(), k, seg.data(), &Praw, d_src.as<int64_t>(),
                                       PD_ALPHABET_AMINO, length_buckets);
    if (st != PD_OK) return st;
    std::unique_ptr<pd_profiles> P(Praw);

    // one all-pairs Best Hit pass and one BBH pass over every job of the chunk
    pdg::QuerySet Q{};
    Q.all_pairs = 1;
    Q.order = P->view.order;
    Q.q0 = 0;
    Q.n_queries = chunk_genes;
    Q.walk = tuning ? tuning->walk : PD_WALK_AUTO;
    C->hits.ctx = c;
    C->hits.all_pairs = 1;
    if ((st = run_hits(c, P.get(), Q, false, &C->hits, 1)) != PD_OK) return st;
    walked += C->hits.walked;
    n_hits_total += C->hits.n_hits;
    pdg::BbhRows R{};
    R.all_pairs = 1;
    R.n_rows = C->hits.n_rows;
    R.gene_genome = P->view.gene_genome;
    R.genome_ptr = P->view.genome_ptr;
    R.row_off = C->hits.row_off.as<unsigned long long>();
    R.row_len = C->hits.row_len.as<uint32_t>();
    R.hit_b = C->hits.out_b.as<uint32_t>();
    if ((st = bbh_impl(c, R, C->hits.out_b.n / sizeof(uint32_t), 0, 0, &C->bbh)) != PD_OK) return st;

    for (uint32_t x = 0; x < cj.size(); ++x) {
      ChunkJob J{};
      J.job = cj[x];
      J.a0 = (uint32_t)cgn[2 * x];
      J.nA = (uint32_t)(cgn[2 * x + 1] - cgn[2 * x]);
      J.b0 = (uint32_t)cgn[2 * x + 1];
      J.nB = (uint32_t)(cgn[2 * x + 2] - cgn[2 * x + 1]);
      J.row0 = row0[cj[x]];
      C->jobs.push_back(J);
    }
    ALLOC(C->d_jobs, sizeof(ChunkJob) * C->jobs.size());
    CK(cudaMemcpyAsync(C->d_jobs.p, C->jobs.data(), sizeof(ChunkJob) * C->jobs.size(), cudaMemcpyHostToDevice,
                       c->stream));
    const uint32_t nj = (uint32_t)C->jobs.size();
    PD_KLAUNCH("batch_rows_len", (k_rows_len<<<grid_of(nj, 1, 152u * 16u), 256, 0, c->stream>>>(
                                      C->d_jobs.as<ChunkJob>(), nj, C->hits.row_len.as<uint32_t>(),
                                      row_len.as<uint32_t>())));
    PD_KLAUNCH("batch_bbh_runs", (k_bbh_runs<<<grid_of(nj, 128, 152u * 4u), 128, 0, c->stream>>>(
                                      C->d_jobs.as<ChunkJob>(), nj, C->bbh.a.as<int32_t>(), (uint32_t)C->bbh.n,
                                      job_cnt.as<uint32_t>())));
    CK(cudaStreamSynchronize(c->stream));  // host staging vectors and the source offsets are released next
    chunks.push_back(std::move(C));
  }

  // ---- assemble: rows and BBH pairs in job order
  CK(pdg::scan_u32_to_u64(&c->L, row_len.as<uint32_t>(), n_rows, B->row_ptr.as<unsigned long long>(), tmp.p,
                          c->stream));
  CK(pdg::scan_u32_to_u64(&c->L, job_cnt.as<uint32_t>(), n_jobs, B->job_ptr.as<unsigned long long>(), tmp.p,
                          c->stream));
  unsigned long long tot[2] = {0, 0};
  CK(cudaMemcpyAsync(&tot[0], B->row_ptr.as<unsigned long long>() + n_rows, sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&tot[1], B->job_ptr.as<unsigned long long>() + n_jobs, sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (tot[0] != n_hits_total) return fail(c, PD_ERR_INTERNAL, "batch Best Hit count mismatch");
  ALLOC(B->cols, sizeof(int32_t) * std::max<unsigned long long>(tot[0], 1));
  ALLOC(B->s, sizeof(uint32_t) * std::max<unsigned long long>(tot[0], 1));
  ALLOC(B->a, sizeof(int32_t) * std::max<unsigned long long>(tot[1], 1));
  ALLOC(B->b, sizeof(int32_t) * std::max<unsigned long long>(tot[1], 1));
  for (auto& C : chunks) {
    const uint32_t nj = (uint32_t)C->jobs.size();
    PD_KLAUNCH("batch_rows_fill",
               (k_rows_fill<<<grid_of(nj, 1, 152u * 16u), 256, 0, c->stream>>>(
                   C->d_jobs.as<ChunkJob>(), nj, C->hits.row_off.as<unsigned long long>(),
                   C->hits.row_len.as<uint32_t>(), C->hits.out_b.as<uint32_t>(), C->hits.out_s.as<uint32_t>(),
                   B->row_ptr.as<unsigned long long>(), B->cols.as<int32_t>(), B->s.as<uint32_t>())));
    PD_KLAUNCH("batch_bbh_fill", (k_bbh_fill<<<grid_of(nj, 1, 152u * 16u), 256, 0, c->stream>>>(
                                      C->d_jobs.as<ChunkJob>(), nj, C->bbh.a.as<int32_t>(), C->bbh.b.as<int32_t>(),
                                      B->job_ptr.as<unsigned long long>(), B->a.as<int32_t>(),
                                      B->b.as<int32_t>())));
  }
  CK(cudaStreamSynchronize(c->stream));  // chunk results are released on return
  pd_batch_info& in = B->info;
  in.n_jobs = n_jobs;
  in.n_chunks = (uint32_t)chunks.size();
  in.n_rows = n_rows;
  in.n_hits = tot[0];
  in.n_bbh = tot[1];
  in.postings_walked = walked;
  *out = B.release();
  return PD_OK;
}

// ---------------------------------------------------------------- genome pairs of one profile set
// One pair job of pd_bbh_pairs: its rows are queries row0 .. row0+nA-1 (genes
// of A, targets B) then row0+nA .. row0+nA+nB-1 (genes of B, targets A).
struct PairJob {
  uint32_t row0, nA, nB, A0, B0;
};

__device__ __forceinline__ bool row_has(const uint32_t* __restrict__ hit_b, unsigned long long off, uint32_t n,
                                        uint32_t a) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (hit_b[off + mid] < a) lo = mid + 1; else hi = mid;
  }
  return lo < n && hit_b[off + lo] == a;
}

__device__ __forceinline__ uint32_t job_of_row(const PairJob* __restrict__ jobs, uint32_t n_jobs, uint32_t r) {
  uint32_t lo = 0, hi = n_jobs;  // last job with row0 <= r
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (jobs[mid].row0 <= r) lo = mid; else hi = mid;
  }
  return lo;
}

// Rows into the batch CSR (columns made local to the partner genome).
__global__ void k_pairs_rows_fill(const PairJob* __restrict__ jobs, uint32_t n_jobs, uint32_t n_rows,
                                  const unsigned long long* __restrict__ row_off, const uint32_t* __restrict__ row_len,
                                  const uint32_t* __restrict__ hit_b, const uint32_t* __restrict__ hit_s,
                                  const unsigned long long* __restrict__ batch_ptr, int32_t* __restrict__ cols,
                                  uint32_t* __restrict__ s) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rows; r += warps) {
    const PairJob J = jobs[job_of_row(jobs, n_jobs, r)];
    const uint32_t partner0 = r < J.row0 + J.nA ? J.B0 : J.A0;
    const unsigned long long src = row_off[r], dst = batch_ptr[r];
    for (uint32_t i = lane; i < row_len[r]; i += 32) {
      cols[dst + i] = (int32_t)(hit_b[src + i] - partner0);
      s[dst + i] = hit_s[src + i];
    }
  }
}

// Mutual check, warp per row of an A genome: b's own row lists a?
__global__ void k_pairs_bbh(const PairJob* __restrict__ jobs, uint32_t n_jobs, uint32_t n_rows,
                            const unsigned long long* __restrict__ row_off, const uint32_t* __restrict__ row_len,
                            const uint32_t* __restrict__ hit_b, const uint32_t* __restrict__ start,
                            uint32_t* __restrict__ cnt, int32_t* __restrict__ pa, int32_t* __restrict__ pb) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rows; r += warps) {
    const PairJob J = jobs[job_of_row(jobs, n_jobs, r)];
    uint32_t n = 0;
    if (r < J.row0 + J.nA) {
      const uint32_t a = J.A0 + (r - J.row0);
      const unsigned long long off = row_off[r];
      const uint32_t len = row_len[r];
      uint32_t pos = start ? start[r] : 0u;
      for (uint32_t e0 = 0; e0 < len; e0 += 32) {
        const uint32_t e = e0 + lane;
        bool f = false;
        uint32_t b = 0;
        if (e < len) {
          b = hit_b[off + e];
          const uint32_t rb = J.row0 + J.nA + (b - J.B0);
          f = row_has(hit_b, row_off[rb], row_len[rb], a);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, f);
        if (start && f) {
          const uint32_t at = pos + (uint32_t)__popc(m & ((1u << lane) - 1u));
          pa[at] = (int32_t)(a - J.A0);
          pb[at] = (int32_t)(b - J.B0);
        }
        pos += (uint32_t)__popc(m);
        n += (uint32_t)__popc(m);
      }
    }
    if (!start && lane == 0) cnt[r] = n;
  }
}

pd_status pairs_impl(pd_ctx* c, const pd_profiles* P, const uint32_t* jobs, uint32_t n_jobs, pd_batch** out) {
  if (n_jobs && !jobs) return fail(c, PD_ERR_ARG, "null jobs");
  if (n_jobs && is_device_ptr(jobs)) return fail(c, PD_ERR_ARG, "jobs must be a host array");
  CK(cudaSetDevice(c->device));
  const auto& gp = P->h_genome_ptr;
  const uint32_t n_genomes = P->view.n_genomes;
  std::vector<PairJob> pj(n_jobs);
  std::vector<uint32_t> qg, qt0, qt1;
  uint32_t row = 0;
  for (uint32_t j = 0; j < n_jobs; ++j) {
    const uint32_t A = jobs[2 * j], B = jobs[2 * j + 1];
    if (A >= n_genomes || B >= n_genomes || A == B)
      return fail(c, PD_ERR_ARG, "job " + std::to_string(j) + " needs two distinct genome indices < n_genomes");
    PairJob J{row, (uint32_t)(gp[A + 1] - gp[A]), (uint32_t)(gp[B + 1] - gp[B]), (uint32_t)gp[A], (uint32_t)gp[B]};
    pj[j] = J;
    for (uint32_t i = 0; i < J.nA; ++i) {
      qg.push_back(J.A0 + i);
      qt0.push_back((uint32_t)gp[B]);
      qt1.push_back((uint32_t)gp[B + 1]);
    }
    for (uint32_t i = 0; i < J.nB; ++i) {
      qg.push_back(J.B0 + i);
      qt0.push_back((uint32_t)gp[A]);
      qt1.push_back((uint32_t)gp[A + 1]);
    }
    row += J.nA + J.nB;
  }
  const uint32_t n_q = row;
  std::unique_ptr<pd_batch> Bt(new pd_batch());
  Bt->ctx = c;
  Buf d_jobs, d_qg, d_t0, d_t1, tmp, cnt, start;
  ALLOC(d_jobs, sizeof(PairJob) * std::max<uint32_t>(n_jobs, 1));
  ALLOC(d_qg, sizeof(uint32_t) * std::max<uint32_t>(n_q, 1));
  ALLOC(d_t0, sizeof(uint32_t) * std::max<uint32_t>(n_q, 1));
  ALLOC(d_t1, sizeof(uint32_t) * std::max<uint32_t>(n_q, 1));
  ALLOC(Bt->row_ptr, sizeof(unsigned long long) * (n_q + 1));
  ALLOC(Bt->job_ptr, sizeof(unsigned long long) * (n_jobs + 1));
  ALLOC(tmp, pdg::scan_temp_bytes(n_q + 1) + 64);
  ALLOC(cnt, sizeof(uint32_t) * std::max<uint32_t>(n_q, 1));
  ALLOC(start, sizeof(uint32_t) * (n_q + 1));
  if (n_jobs) CK(cudaMemcpyAsync(d_jobs.p, pj.data(), sizeof(PairJob) * n_jobs, cudaMemcpyHostToDevice, c->stream));
  if (n_q) {
    CK(cudaMemcpyAsync(d_qg.p, qg.data(), sizeof(uint32_t) * n_q, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(d_t0.p, qt0.data(), sizeof(uint32_t) * n_q, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(d_t1.p, qt1.data(), sizeof(uint32_t) * n_q, cudaMemcpyHostToDevice, c->stream));
  }
  // one sum-min / Best Hit launch sequence over every query of every job
  pd_hits H;
  H.ctx = c;
  pdg::QuerySet Q{};
  Q.all_pairs = 0;
  Q.n_queries = n_q;
  Q.q_gene = d_qg.as<uint32_t>();
  Q.q_t0 = d_t0.as<uint32_t>();
  Q.q_t1 = d_t1.as<uint32_t>();
  pd_status st = run_hits(c, P, Q, false, &H, 1);
  if (st != PD_OK) return st;
  CK(pdg::scan_u32_to_u64(&c->L, H.row_len.as<uint32_t>(), n_q, Bt->row_ptr.as<unsigned long long>(), tmp.p,
                          c->stream));
  if (n_q)
    PD_KLAUNCH("pairs_bbh_count", (k_pairs_bbh<<<grid_of((uint64_t)n_q * 32, 256, 152u * 16u), 256, 0, c->stream>>>(
                                       d_jobs.as<PairJob>(), n_jobs, n_q, H.row_off.as<unsigned long long>(),
                                       H.row_len.as<uint32_t>(), H.out_b.as<uint32_t>(), nullptr,
                                       cnt.as<uint32_t>(), nullptr, nullptr)));
  CK(pdg::scan_u32(&c->L, cnt.as<uint32_t>(), n_q, start.as<uint32_t>(), tmp.p, c->stream));
  unsigned long long n_hits = 0;
  uint32_t n_bbh = 0;
  std::vector<uint32_t> h_start(n_q + 1);
  CK(cudaMemcpyAsync(&n_hits, Bt->row_ptr.as<unsigned long long>() + n_q, sizeof(n_hits), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaMemcpyAsync(h_start.data(), start.p, sizeof(uint32_t) * (n_q + 1), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  n_bbh = h_start[n_q];
  std::vector<unsigned long long> job_ptr(n_jobs + 1);
  for (uint32_t j = 0; j < n_jobs; ++j) job_ptr[j] = h_start[pj[j].row0];
  job_ptr[n_jobs] = n_bbh;
  CK(cudaMemcpyAsync(Bt->job_ptr.p, job_ptr.data(), sizeof(unsigned long long) * (n_jobs + 1),
                     cudaMemcpyHostToDevice, c->stream));
  ALLOC(Bt->cols, sizeof(int32_t) * std::max<unsigned long long>(n_hits, 1));
  ALLOC(Bt->s, sizeof(uint32_t) * std::max<unsigned long long>(n_hits, 1));
  ALLOC(Bt->a, sizeof(int32_t) * std::max<uint32_t>(n_bbh, 1));
  ALLOC(Bt->b, sizeof(int32_t) * std::max<uint32_t>(n_bbh, 1));
  if (n_q) {
    PD_KLAUNCH("pairs_rows_fill",
               (k_pairs_rows_fill<<<grid_of((uint64_t)n_q * 32, 256, 152u * 16u), 256, 0, c->stream>>>(
                   d_jobs.as<PairJob>(), n_jobs, n_q, H.row_off.as<unsigned long long>(), H.row_len.as<uint32_t>(),
                   H.out_b.as<uint32_t>(), H.out_s.as<uint32_t>(), Bt->row_ptr.as<unsigned long long>(),
                   Bt->cols.as<int32_t>(), Bt->s.as<uint32_t>())));
    if (n_bbh)
      PD_KLAUNCH("pairs_bbh_write",
                 (k_pairs_bbh<<<grid_of((uint64_t)n_q * 32, 256, 152u * 16u), 256, 0, c->stream>>>(
                     d_jobs.as<PairJob>(), n_jobs, n_q, H.row_off.as<unsigned long long>(), H.row_len.as<uint32_t>(),
                     H.out_b.as<uint32_t>(), start.as<uint32_t>(), nullptr, Bt->a.as<int32_t>(),
                     Bt->b.as<int32_t>())));
  }
  CK(cudaStreamSynchronize(c->stream));  // temporaries and the hits are released on return
  pd_batch_info& in = Bt->info;
  in.n_jobs = n_jobs;
  in.n_chunks = 1;
  in.n_rows = n_q;
  in.n_hits = n_hits;
  in.n_bbh = n_bbh;
  in.postings_walked = H.walked;
  *out = Bt.release();
  return PD_OK;
}

}  // namespace

PD_API pd_status pd_bbh_pairs(pd_ctx* c, const pd_profiles* P, const uint32_t* jobs, uint32_t n_jobs,
                              pd_batch** out) {
  PhaseRange range_("pd: bbh of listed pairs");
  if (!c || !P || !out) return PD_ERR_ARG;
  *out = nullptr;
  try {
    return pairs_impl(c, P, jobs, n_jobs, out);
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_bbh_pairs");
  }
}

PD_API pd_status pd_bbh_batch(pd_ctx* c, const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr,
                              uint32_t n_genes, const int32_t* genome_ptr, uint32_t n_genomes, const uint32_t* jobs,
                              const int32_t* job_k, uint32_t n_jobs, const pd_batch_tuning* tuning, pd_batch** out) {
  PhaseRange range_("pd: batch");
  if (!c || !out) return PD_ERR_ARG;
  *out = nullptr;
  try {
    return batch_impl(c, residues, n_res, gene_ptr, n_genes, genome_ptr, n_genomes, jobs, job_k, n_jobs, tuning,
                      out);
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_bbh_batch");
  }
}

PD_API pd_status pd_batch_autotune(pd_ctx* c, const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr,
                                   uint32_t n_genes, const int32_t* genome_ptr, uint32_t n_genomes,
                                   const uint32_t* jobs, const int32_t* job_k, uint32_t n_jobs, uint32_t n_sample,
                                   pd_batch_tuning* best, double* ms_per_job) {
  if (!c || !best) return PD_ERR_ARG;
  try {
    CK(cudaSetDevice(c->device));
    const uint32_t ns = std::min<uint32_t>(n_jobs, n_sample ? n_sample : 100u);
    if (ns == 0) return fail(c, PD_ERR_ARG, "no jobs to sample");
    std::vector<pd_batch_tuning> cand;
    for (uint32_t order : {0u, 1u})
      for (uint64_t w : {1ull << 28, 1ull << 29})
        for (uint32_t j : {8u, 32u, 0u}) cand.push_back(pd_batch_tuning{w, j, order, PD_WALK_AUTO});
    // after the chunking and order candidates: the fastest of them with each
    // explicit posting walk (the automatic choice is one of the two)
    const size_t n_first = cand.size();
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = -1.f;
    pd_status st = PD_OK;
    for (size_t x = 0; st == PD_OK; ++x) {
      if (x == n_first && best_ms >= 0.f)
        for (uint32_t walk : {PD_WALK_MERGE, PD_WALK_WARP}) {
          pd_batch_tuning t = *best;
          t.walk = walk;
          cand.push_back(t);
        }
      if (x >= cand.size()) break;
      for (int rep = 0; rep < 2 && st == PD_OK; ++rep) {  // one warm-up, one timed run
        pd_batch* B = nullptr;
        if (cudaEventRecord(e0, c->stream) != cudaSuccess) st = fail_cuda(c, cudaGetLastError(), "event");
        if (st == PD_OK)
          st = batch_impl(c, residues, n_res, gene_ptr, n_genes, genome_ptr, n_genomes, jobs, job_k, ns, &cand[x],
                          &B);
        if (st == PD_OK && cudaEventRecord(e1, c->stream) != cudaSuccess)
          st = fail_cuda(c, cudaGetLastError(), "event");
        if (st == PD_OK && cudaEventSynchronize(e1) != cudaSuccess) st = fail_cuda(c, cudaGetLastError(), "event");
        float ms = 0.f;
        if (st == PD_OK && rep == 1 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            (best_ms < 0.f || ms < best_ms)) {
          best_ms = ms;
          *best = cand[x];
        }
        pd_batch_free(B);
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PD_OK) return st;
    if (ms_per_job) *ms_per_job = best_ms / ns;
    return PD_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_batch_autotune");
  }
}

PD_API pd_status pd_batch_get_info(const pd_batch* B, pd_batch_info* info) {
  if (!B || !info) return PD_ERR_ARG;
  *info = B->info;
  return PD_OK;
}

PD_API pd_status pd_batch_copy_hits(pd_ctx* c, const pd_batch* B, int64_t* row_ptr, int32_t* cols, uint32_t* s) {
  if (!c || !B) return PD_ERR_ARG;
  try {
    CK(cudaSetDevice(c->device));
    pd_status st;
    if ((st = copy_out(c, row_ptr, B->row_ptr.p, sizeof(int64_t) * (B->info.n_rows + 1))) != PD_OK) return st;
    if ((st = copy_out(c, cols, B->cols.p, sizeof(int32_t) * B->info.n_hits)) != PD_OK) return st;
    if ((st = copy_out(c, s, B->s.p, sizeof(uint32_t) * B->info.n_hits)) != PD_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    return PD_OK;
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_batch_copy_hits");
  }
}

PD_API pd_status pd_batch_copy_bbh(pd_ctx* c, const pd_batch* B, int64_t* job_ptr, int32_t* a, int32_t* b) {
  if (!c || !B) return PD_ERR_ARG;
  try {
    CK(cudaSetDevice(c->device));
    pd_status st;
    if ((st = copy_out(c, job_ptr, B->job_ptr.p, sizeof(int64_t) * (B->info.n_jobs + 1))) != PD_OK) return st;
    if ((st = copy_out(c, a, B->a.p, sizeof(int32_t) * B->info.n_bbh)) != PD_OK) return st;
    if ((st = copy_out(c, b, B->b.p, sizeof(int32_t) * B->info.n_bbh)) != PD_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    return PD_OK;
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_batch_copy_bbh");
  }
}

PD_API void pd_batch_free(pd_batch* B) { delete B; }
