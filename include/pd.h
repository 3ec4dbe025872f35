/*
 * pd.h -- C ABI of the GB300 PanDelos-plus hot path (libpandelos_gpu.so).
 *
 * The library computes, for genomes made of amino-acid genes:
 *   - per-gene k-mer multiplicity vectors (Eqs. (1)-(3), Algorithm 1);
 *   - for every cross-genome gene pair (a, b) the exact integer numerator of
 *     the generalized Jaccard similarity, s = sum over shared k-mers of
 *     min(mult_a, mult_b), whose denominator is La + Lb - s (Eq. (5); La is the
 *     number of k-mer windows of a);
 *   - Best Hits: for a gene a and a target genome G_j, all genes of G_j whose
 *     similarity to a equals the maximum (Eq. (8), Algorithm 2);
 *   - Bidirectional Best Hits: pairs (a, b) with b in BH(a, G_j) and a in
 *     BH(b, G_i) (Eq. (9), Algorithm 3).
 *
 * Conventions shared by every call:
 *   - Every call returns a pd_status; no C++ exception crosses this ABI.
 *     On failure pd_last_error(ctx) holds a one-line message.
 *   - Inputs may live in host or device memory (detected per pointer); the
 *     library copies host inputs to the device on the context's stream.
 *   - Handles (pd_profiles, pd_hits, pd_bbh_set) own device memory obtained
 *     from the context's allocator until the matching *_free call.  A handle
 *     must be freed before its context is destroyed.  Caller buffers are only
 *     borrowed for the duration of a call.
 *   - All work of one context runs on its CUDA stream.  Calls that produce
 *     data-dependent sizes synchronize that stream before they return.  One
 *     context must not be used by two host threads at once.
 *   - Gene indices: inside a dataset genes are numbered 0..n_genes-1 in input
 *     order ("global" ids); genome i holds the contiguous genes
 *     genome_ptr[i] .. genome_ptr[i+1]-1.  Per-pair results use "local"
 *     indices (position inside the genome).
 *   - Exactness: every value is an integer; ratios s1/d1 and s2/d2 are
 *     compared by 64-bit cross-multiplication, so ties are exact.
 *   - Candidates: a pair with s = 0 is never a hit (a minimum k-mer overlap is
 *     required, "PanDelos methodology"); a gene with no candidate in G_j has an
 *     empty Best Hit set, and a gene shorter than k never hits.
 */
#ifndef PD_H_
#define PD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PD_OK = 0,
  PD_ERR_ARG = 1,            /* invalid pointer, size, index, range or handle */
  PD_ERR_ALPHABET = 2,       /* a residue is not one of ACDEFGHIKLMNPQRSTVWY */
  PD_ERR_GENE_TOO_LONG = 3,  /* a gene has more than PD_MAX_WINDOWS k-mer windows */
  PD_ERR_K_RANGE = 4,        /* k outside [1, PD_MAX_K] */
  PD_ERR_OOM = 5,            /* the allocator returned NULL */
  PD_ERR_BUDGET = 6,         /* over a stated memory budget or fixed limit (served index, segmented build, no-alloc call) */
  PD_ERR_CUDA = 7,           /* a CUDA runtime call or kernel launch failed */
  PD_ERR_TIMEOUT = 8,        /* a bounded wait expired (pd_index_poll) */
  PD_ERR_BUSY = 9,           /* no free slot (the served index would exceed PD_MAX_GENOMES) */
  PD_ERR_INTERNAL = 10       /* an internal invariant failed (a bug) */
} pd_status;

/* Alphabets ("nucleotide or amino acid", Basic notions). */
#define PD_ALPHABET_AMINO 20      /* ACDEFGHIKLMNPQRSTVWY */
#define PD_ALPHABET_NUCLEOTIDE 4  /* ACGT */
/* Largest k: the k-mer dictionary is a bitmap over all |alphabet|^k codes. */
#define PD_MAX_K 8
#define PD_MAX_K_NUCLEOTIDE 16
/* Largest number of windows (|g| - k + 1) of one gene: counts are 16-bit. */
#define PD_MAX_WINDOWS 65535u
/* Largest number of genomes in one dataset (per-genome maxima live in shared memory). */
#define PD_MAX_GENOMES 4096u

typedef struct pd_ctx pd_ctx;
typedef struct pd_profiles pd_profiles;
typedef struct pd_hits pd_hits;
typedef struct pd_bbh_set pd_bbh_set;

/* Device allocator hooks.  alloc returns a device pointer usable on `stream`
 * (aligned to at least 256 bytes) or NULL; free releases it.  Passing NULL
 * hooks gives the context a CUDA memory pool of its own (stream-ordered
 * allocation, freed memory kept for reuse until the context is destroyed). */
typedef void* (*pd_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*pd_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context; on failure *out is NULL. */
pd_status pd_ctx_create(int device, void* cuda_stream, pd_alloc_fn alloc, pd_free_fn free_fn,
                        void* user, pd_ctx** out);
/* Destroy a context (synchronizes its stream).  NULL is ignored. */
void pd_ctx_destroy(pd_ctx* ctx);
/* Replace the stream used by later calls. */
pd_status pd_ctx_set_stream(pd_ctx* ctx, void* cuda_stream);
/* Last error message of this context ("" if none); owned by the context. */
const char* pd_last_error(const pd_ctx* ctx);
/* Number of kernels this library has launched through `ctx` so far. */
uint64_t pd_ctx_launch_count(const pd_ctx* ctx);
/* Per-kernel device timing.  When enabled, every launch is bracketed by CUDA
 * events recorded on the launching stream.  pd_ctx_kernel_time synchronizes
 * the stream and returns the summed milliseconds and launch count of kernel
 * `name` since the last reset (name = NULL: all kernels). */
pd_status pd_ctx_set_timing(pd_ctx* ctx, int enable);
/* Restrict the timing above to launches of kernel `name` (NULL or "": every
 * kernel, the default), so that a timed region pays for the events of one
 * kernel only.  The name is copied. */
pd_status pd_ctx_set_timing_filter(pd_ctx* ctx, const char* name);
pd_status pd_ctx_kernel_time(pd_ctx* ctx, const char* name, double* ms, uint64_t* launches);
pd_status pd_ctx_reset_timing(pd_ctx* ctx);

/* ---------------------------------------------------------------- k rule */

/* Eq. (4), "Basic notions": k = log_|Gamma| of the dataset size.  Read as the
 * smallest integer k >= 1 with alphabet^k >= total_residues (exact integer
 * powers).  Returns -1 if alphabet < 2. */
int pd_choose_k(uint64_t total_residues, int alphabet);

/* ---------------------------------------------------------------- profiles */

/* Build the k-mer profiles of a dataset ("Multiplicity vector building
 * phase", Algorithm 1; steps: residue mapping, rolling base-20 k-mer codes,
 * dictionary of distinct codes -> dense ids, per-gene sorted (id, count)
 * vectors, and the inverted index id -> (gene, count) postings).
 *   residues   n_res bytes, all genes concatenated, letters ACDEFGHIKLMNPQRSTVWY
 *   gene_ptr   n_genes+1 int64: gene g is residues[gene_ptr[g] .. gene_ptr[g+1])
 *              (gene_ptr[0] = 0, non-decreasing, gene_ptr[n_genes] = n_res)
 *   genome_ptr n_genomes+1 int32: genome i holds genes genome_ptr[i] ..
 *              genome_ptr[i+1]-1 (genome_ptr[0] = 0, non-decreasing,
 *              genome_ptr[n_genomes] = n_genes)
 *   k          1..PD_MAX_K
 * Errors: PD_ERR_ALPHABET (a byte outside the alphabet), PD_ERR_GENE_TOO_LONG,
 * PD_ERR_K_RANGE, PD_ERR_ARG (malformed offsets, n_genomes > PD_MAX_GENOMES,
 * more than 2^32-1 windows in total), PD_ERR_OOM, PD_ERR_CUDA.
 * *out receives a device-resident handle. */
pd_status pd_build_profiles(pd_ctx* ctx, const uint8_t* residues, uint64_t n_res,
                            const int64_t* gene_ptr, uint32_t n_genes, const int32_t* genome_ptr,
                            uint32_t n_genomes, int k, pd_profiles** out);

/* pd_build_profiles over an alphabet of PD_ALPHABET_AMINO (20, k <= PD_MAX_K)
 * or PD_ALPHABET_NUCLEOTIDE (4: ACGT, k <= PD_MAX_K_NUCLEOTIDE) letters; every
 * later call is the same for either alphabet.  pd_build_profiles is this call
 * with the amino-acid alphabet.  Codes returned by the copy calls are base-4
 * for nucleotides. */
pd_status pd_build_profiles_alphabet(pd_ctx* ctx, const uint8_t* residues, uint64_t n_res,
                                     const int64_t* gene_ptr, uint32_t n_genes, const int32_t* genome_ptr,
                                     uint32_t n_genomes, int alphabet, int k, pd_profiles** out);

/* pd_build_profiles over several independent problems at once.  genome_seg
 * (HOST array, n_genomes entries, each < n_genomes) assigns every genome to a
 * segment; k-mers of different segments are different dictionary entries
 * (the segment is part of the k-mer's identity), so genes of different
 * segments share no k-mer, have sum-min 0 and are never candidates (reading
 * of "minimum overlap" under Eq. (8)).  Best Hits and BBH of a segmented
 * profile set therefore equal those of each segment profiled alone.  Codes
 * returned by pd_profiles_copy_mv / _copy_index are segment * 20^k + code.
 * Extra error: PD_ERR_BUDGET when (max segment + 1) * 20^k bits exceed the
 * 4 GiB dictionary bitmap limit. */
pd_status pd_build_profiles_segmented(pd_ctx* ctx, const uint8_t* residues, uint64_t n_res,
                                      const int64_t* gene_ptr, uint32_t n_genes, const int32_t* genome_ptr,
                                      uint32_t n_genomes, const uint32_t* genome_seg, int k,
                                      pd_profiles** out);

typedef struct {
  int k;
  uint32_t n_genes, n_genomes;
  uint64_t n_windows;   /* sum of La over genes */
  uint64_t n_distinct;  /* distinct k-mers of the dataset (dictionary size D) */
  uint64_t n_entries;   /* sum over genes of distinct k-mers (MV entries = postings) */
  uint32_t max_posting; /* longest posting list */
  uint32_t count_bits;  /* bits of the count field in a packed posting */
  uint64_t device_bytes;/* device memory held by the handle */
  int alphabet;         /* 20 or 4 */
  uint64_t n_join;      /* postings the all-against-all Best Hit walk visits: the sum over MV entries of
                           their k-mer's posting-list length (the sum over k-mers of length squared) */
} pd_profiles_info;

pd_status pd_profiles_get_info(const pd_profiles* prof, pd_profiles_info* info);
/* The genome offsets the profiles were built with: n_genomes+1 int32 into a
 * HOST buffer (genome i holds genes genome_ptr[i] .. genome_ptr[i+1]-1). */
pd_status pd_profiles_genome_ptr(const pd_profiles* prof, int32_t* genome_ptr);

/* Copy the multiplicity vector of every gene (test and inspection hook).
 *   mv_ptr  n_genes+1 int64 (CSR offsets), codes n_entries uint64 (base-20
 *   k-mer code, first letter most significant, letters numbered in the order
 *   ACDEFGHIKLMNPQRSTVWY), counts n_entries uint32, La n_genes uint32.
 * Each gene's entries are in ascending code order.  Any pointer may be NULL
 * to skip that array; pointers may be host or device. */
pd_status pd_profiles_copy_mv(pd_ctx* ctx, const pd_profiles* prof, int64_t* mv_ptr,
                              uint64_t* codes, uint32_t* counts, uint32_t* La);

/* Copy the inverted index (test and inspection hook): for each distinct
 * k-mer in ascending code order, its postings (gene, count) in ascending
 * gene order.  post_ptr n_distinct+1 int64, codes n_distinct uint64,
 * genes n_entries int32, counts n_entries uint32.  NULL skips an array. */
pd_status pd_profiles_copy_index(pd_ctx* ctx, const pd_profiles* prof, int64_t* post_ptr,
                                 uint64_t* codes, int32_t* genes, uint32_t* counts);

void pd_profiles_free(pd_profiles* prof);

/* ---------------------------------------------------------------- hits */

/* Best Hits of every gene against every other genome of the dataset
 * (all-against-all, "PanDelos-plus pipeline overview" phase (b) for all
 * genome pairs at once).  Row a of the result lists, for every genome j other
 * than a's own, the global ids of BH(a, G_j) (Eq. (8)); rows are grouped by
 * target genome because global ids are contiguous per genome, and ascending. */
pd_status pd_best_hits_all(pd_ctx* ctx, const pd_profiles* prof, pd_hits** out);

/* How pd_best_hits_all covers the genome pairs (no counterpart in the paper;
 * the results are identical either way).  enable != 0 (the default): the
 * similarity is symmetric (Eq. (5)), so each unordered genome pair is walked
 * from one side -- a query gene walks only the genomes after its own, emits
 * its Best Hits there and keeps, for every target, the best ratio over the
 * query's genome (the reverse direction, the column maximum of Algorithm 3);
 * used while genes x genomes x 8 bytes stay within 4 GiB.  enable == 0: every
 * query walks every other genome.  Errors: PD_ERR_ARG (null context). */
pd_status pd_ctx_set_symmetric(pd_ctx* ctx, int enable);

/* Posting walk of the sum-min kernel (no counterpart in the paper; results
 * are identical for every choice, only the time differs).  A query's staged
 * posting lists are read either by the merge-path walk (each thread a run of
 * consecutive postings, batches of four) or by the warp-cooperative walk
 * (each warp 32 consecutive postings per round; suits long lists).
 * PD_WALK_AUTO (the default) takes the warp walk when the build's join
 * (pd_profiles_info.n_join) is at least 16 postings per vector entry and the
 * postings take at least 512 MB (smaller indexes stay close enough to L2
 * for the merge-path walk).
 * Applies to every later Best Hit call on the context.  Errors: PD_ERR_ARG
 * (null context, unknown mode). */
#define PD_WALK_AUTO 0u
#define PD_WALK_MERGE 1u
#define PD_WALK_WARP 2u
pd_status pd_ctx_set_walk(pd_ctx* ctx, uint32_t mode);

/* One shard of pd_best_hits_all, for splitting one dataset's all-against-all
 * work across processes or GPUs that each hold the same profiles.  The paper
 * decomposes phase (b) by data, one query gene (a row of Algorithm 2) being
 * one unit of work ("Parallel implementation"); here shard `shard` of
 * `n_shards` takes the query genes g with g mod n_shards == shard (genes of
 * every genome and length, so shards get similar work, and the same shards
 * whichever process built the profiles).  The result has a row
 * for every gene (as pd_best_hits_all); rows of genes outside the shard are
 * empty.  The union over shard = 0 .. n_shards-1 of the rows equals
 * pd_best_hits_all exactly.  Errors: PD_ERR_ARG (n_shards 0, shard >=
 * n_shards), PD_ERR_OOM, PD_ERR_CUDA. */
pd_status pd_best_hits_shard(pd_ctx* ctx, const pd_profiles* prof, uint32_t shard, uint32_t n_shards,
                             pd_hits** out);

/* A Best Hit result assembled from pieces -- typically the shards of
 * pd_best_hits_shard gathered from other processes or GPUs -- as one handle
 * that pd_bbh_all and pd_hits_copy accept.  Piece p is a CSR over every gene:
 * row_ptr[p] n_genes+1 int64 from 0 to n_hits[p]; cols[p] n_hits[p] int32
 * global gene ids, strictly ascending inside a row and outside the row's own
 * genome; s[p] n_hits[p] uint32 sum-min.  A gene's row may be non-empty in at
 * most one piece (the merged row is that one).  Host or device pointers,
 * copied before return.  Errors: PD_ERR_ARG (a malformed piece, or a row in
 * two pieces), PD_ERR_OOM, PD_ERR_CUDA. */
pd_status pd_hits_import(pd_ctx* ctx, const pd_profiles* prof, uint32_t n_pieces, const int64_t* const* row_ptr,
                         const int32_t* const* cols, const uint32_t* const* s, const uint64_t* n_hits,
                         pd_hits** out);

/* Best Hits BH(a, G_gj) of every gene a of genome gi (Algorithm 2 for one
 * genome pair).  Rows are the genes of G_gi (local), columns local to G_gj.
 * gi == gj is PD_ERR_ARG. */
pd_status pd_best_hits(pd_ctx* ctx, const pd_profiles* prof, uint32_t gi, uint32_t gj,
                       pd_hits** out);

typedef struct {
  uint32_t n_rows;      /* number of query genes */
  uint64_t n_hits;      /* total Best Hit entries */
  uint32_t row_base;    /* global id of row 0 (pair form), 0 for the all form */
  uint32_t col_base;    /* global id subtracted from columns (pair form), 0 for all */
  uint32_t n_deferred;  /* rows that took the large-accumulator path */
  uint64_t postings_walked; /* (query k-mer, posting) matches visited */
} pd_hits_info;

pd_status pd_hits_get_info(const pd_hits* hits, pd_hits_info* info);

/* Copy Best Hits as CSR: row_ptr n_rows+1 int64, cols n_hits int32 (local
 * for the pair form, global for the all form), s n_hits uint32 (the pair's
 * sum-min; its Eq. (5) denominator is La + Lb - s).  NULL skips an array;
 * pointers may be host or device.  *n_hits (if not NULL) receives the count. */
pd_status pd_hits_copy(pd_ctx* ctx, const pd_hits* hits, int64_t* row_ptr, int32_t* cols,
                       uint32_t* s, uint64_t* n_hits);
void pd_hits_free(pd_hits* hits);

/* ---------------------------------------------------------------- BBH */

/* Bidirectional Best Hits of all genome pairs from an all-against-all
 * Best Hit result (Eq. (9), Algorithm 3).  Pairs (a, b) are global ids with
 * genome(a) < genome(b), in ascending (a, b) order. */
pd_status pd_bbh_all(pd_ctx* ctx, const pd_profiles* prof, const pd_hits* hits, pd_bbh_set** out);

/* Bidirectional Best Hits of one genome pair (gi, gj), gi != gj: both Best
 * Hit directions and the mutual check.  Pairs (a, b) are local (a in G_gi,
 * b in G_gj), ascending. */
pd_status pd_bbh(pd_ctx* ctx, const pd_profiles* prof, uint32_t gi, uint32_t gj, pd_bbh_set** out);

/* Candidate filters of Eqs. (6) and (7), applied before the Best Hit argmax:
 * a pair (a, b) with s >= 1 stays a candidate only if
 *   theta: |a| * theta_den >= theta_num * |b| and |b| * theta_den >= theta_num * |a|
 *          (gene lengths in letters, Eq. (6));
 *   tau:   p_k(a -> b) >= tau and p_k(b -> a) >= tau, where p_k(a -> b) is the
 *          sum of mult_a(w) over the k-mers w shared with b, divided by
 *          |a| - k + 1 (Eq. (7)), compared exactly as
 *          p_num * tau_den >= tau_num * (|a| - k + 1).
 * theta = theta_num / theta_den and tau = tau_num / tau_den must lie in [0, 1]
 * (den >= 1); a numerator of 0 turns that filter off.  The paper gives no
 * values; both default to off in every other call. */
typedef struct {
  uint32_t theta_num, theta_den;
  uint32_t tau_num, tau_den;
} pd_filter;

/* pd_best_hits_all / pd_best_hits with the candidate filters; the results
 * feed pd_bbh_all / are read with pd_hits_copy like the unfiltered ones. */
pd_status pd_best_hits_all_filtered(pd_ctx* ctx, const pd_profiles* prof, const pd_filter* filter, pd_hits** out);
pd_status pd_best_hits_filtered(pd_ctx* ctx, const pd_profiles* prof, uint32_t gi, uint32_t gj,
                                const pd_filter* filter, pd_hits** out);

/* Within-genome (paralog) Best Hits: Eq. (8) with both genes in the same
 * genome, the gene itself excluded -- BH(a, G_i minus a) for every gene a of
 * every genome G_i, same candidate and tie rules as across genomes.  Rows are
 * all genes, columns global ids; copy with pd_hits_copy. */
pd_status pd_paralog_hits(pd_ctx* ctx, const pd_profiles* prof, pd_hits** out);
/* Mutual within-genome Best Hits of a pd_paralog_hits result (Eq. (9) inside
 * one genome): pairs (a, b), a < b, same genome, ascending. */
pd_status pd_paralog_bbh(pd_ctx* ctx, const pd_profiles* prof, const pd_hits* hits, pd_bbh_set** out);

/* Copy pairs: a and b n_pairs int32 each (host or device, NULL to skip);
 * *n_pairs (if not NULL) receives the count. */
pd_status pd_bbh_copy(pd_ctx* ctx, const pd_bbh_set* set, int32_t* a, int32_t* b, uint64_t* n_pairs);
uint64_t pd_bbh_count(const pd_bbh_set* set);
void pd_bbh_free(pd_bbh_set* set);

/* ---------------------------------------------------------------- families */

/* Connected components of an undirected graph of n_nodes nodes given by
 * n_edges edges (a[e], b[e]) (int32, host or device): label[v] (n_nodes
 * int32, host or device) receives the smallest node id of v's component;
 * *n_components (if not NULL) the number of components.  An edge naming a
 * node outside [0, n_nodes) is PD_ERR_ARG. */
pd_status pd_components(pd_ctx* ctx, const int32_t* a, const int32_t* b, uint64_t n_edges, uint32_t n_nodes,
                        int32_t* label, uint32_t* n_components);
/* Gene families (phase (c), "extract gene families from the Bidirectional
 * Best Hits"): the connected components of the BBH graph of pd_bbh_all, one
 * label per gene (global ids, n_genes of the profiled dataset), each family
 * labelled by its smallest gene id.  The refinement PanDelos applies to the
 * components is not specified by the paper and is not applied. */
pd_status pd_families(pd_ctx* ctx, const pd_bbh_set* bbh, uint32_t n_genes, int32_t* family, uint32_t* n_families);

/* ---------------------------------------------------------------- sum-min */

/* Sum-min of listed gene pairs by the paper's own form: the two
 * multiplicity vectors, sorted by k-mer, walked side by side (the similarity
 * of Algorithm 2; Eq. (5)).  Pair i is (a[i], b[i]), global gene ids of this
 * dataset (any genomes, a gene with itself allowed).  s[i] receives sum-min,
 * den[i] the Eq. (5) denominator sum-max = La + Lb - s; GJ = s / den (0/0 for
 * two genes without windows).  a, b, s, den are host or device pointers (n
 * entries each; s or den NULL to skip).  One warp merges one pair, so the
 * call suits known pairs (the similarity of BBH pairs, a candidate list); the
 * all-against-all search is pd_best_hits_all.  Errors: PD_ERR_ARG (a gene id
 * not below n_genes), PD_ERR_OOM, PD_ERR_CUDA. */
pd_status pd_summin_list(pd_ctx* ctx, const pd_profiles* prof, const uint32_t* a, const uint32_t* b, uint64_t n,
                         uint32_t* s, uint32_t* den);

/* Every pair (a in G_gi, b in G_gj) with s >= 1 and its s (Eq. (5)
 * numerator), local indices, ascending (a, b).  Two-phase: with a == NULL
 * only *n is written; otherwise a, b, s must hold *n entries (host or device)
 * and the call fills them.  Exposes the sum-min step for checking. */
pd_status pd_summin_pairs(pd_ctx* ctx, const pd_profiles* prof, uint32_t gi, uint32_t gj,
                          int32_t* a, int32_t* b, uint32_t* s, uint64_t* n);

/* ---------------------------------------------------------------- batched jobs */

typedef struct pd_batch pd_batch;

/* How a batch is cut into chunks; each chunk is one segmented profile build,
 * one Best Hit launch sequence and one BBH launch sequence over all of its
 * jobs.  Zero fields take the defaults. */
typedef struct {
  uint64_t max_chunk_windows; /* k-mer windows profiled together (default 2^29) */
  uint32_t max_chunk_jobs;    /* jobs per chunk (default: as many as the 256 MiB
                                 chunk dictionary bitmap holds at the job's k,
                                 at most PD_MAX_GENOMES / 2) */
  uint32_t query_order;       /* sum-min work queue: 0 = length buckets (longest
                                 first), min-hash inside a bucket; 1 = min-hash only */
  uint32_t walk;              /* posting walk of the sum-min kernel (PD_WALK_*) */
} pd_batch_tuning;

typedef struct {
  uint32_t n_jobs;
  uint32_t n_chunks;         /* chunks the batch was cut into */
  uint64_t n_rows;           /* sum over jobs of |A| + |B| */
  uint64_t n_hits;           /* Best Hit entries, both directions, all jobs */
  uint64_t n_bbh;            /* BBH pairs, all jobs */
  uint64_t postings_walked;  /* (query k-mer, posting) matches visited */
} pd_batch_info;

/* Best Hits in both directions and Bidirectional Best Hits (Eqs. (8)-(9),
 * Algorithms 2-3) of many independent genome-pair jobs, each at its own k.
 *   residues, gene_ptr, genome_ptr  the genomes, as in pd_build_profiles
 *              (residues host or device; offsets host or device)
 *   jobs       HOST array of 2*n_jobs genome indices: job j compares genome
 *              A = jobs[2j] with genome B = jobs[2j+1] (A != B); a genome may
 *              appear in several jobs
 *   job_k      HOST array of n_jobs k values, each in 1..PD_MAX_K
 *   tuning     NULL for the defaults
 * Jobs with the same k are profiled together in chunks (segmented profiles:
 * one dictionary namespace per job), so one launch sequence serves a whole
 * chunk.  Each job's result equals pd_bbh / pd_best_hits on a dataset of its
 * two genomes alone.  Errors as pd_build_profiles, plus PD_ERR_ARG for bad job
 * entries.  *out receives a device-resident handle. */
pd_status pd_bbh_batch(pd_ctx* ctx, const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr,
                       uint32_t n_genes, const int32_t* genome_ptr, uint32_t n_genomes, const uint32_t* jobs,
                       const int32_t* job_k, uint32_t n_jobs, const pd_batch_tuning* tuning, pd_batch** out);
/* Many genome pairs of ONE profiled dataset (Algorithms 2-3 for each pair),
 * answered by one sum-min / Best Hit launch sequence over the genes of all
 * pairs: jobs is a HOST array of 2*n_jobs genome indices of prof (A != B; a
 * genome may appear in several jobs).  The result has the pd_bbh_batch layout
 * (rows of A then B per job, partner-local columns; BBH pairs per job) and is
 * read with pd_batch_get_info / pd_batch_copy_hits / pd_batch_copy_bbh.
 * Each job equals pd_best_hits(gi=A, gj=B), pd_best_hits(B, A) and
 * pd_bbh(A, B) on the same profiles. */
pd_status pd_bbh_pairs(pd_ctx* ctx, const pd_profiles* prof, const uint32_t* jobs, uint32_t n_jobs,
                       pd_batch** out);
pd_status pd_batch_get_info(const pd_batch* batch, pd_batch_info* info);
/* Autotuner of pd_bbh_batch: runs the first n_sample jobs (0 = min(n_jobs,
 * 100)) once with each candidate tuning (jobs per chunk 8 / 32 / dictionary
 * default, windows per chunk 2^28 / 2^29, both query orders, the automatic
 * walk; then the fastest of these with each explicit posting walk), timed
 * with CUDA events on the context's stream after one warm-up, and writes the
 * fastest to *best (and its time per sampled job, in milliseconds, to
 * *ms_per_job if not NULL).  Results never depend on the tuning, only the
 * time does.  Arguments as pd_bbh_batch. */
pd_status pd_batch_autotune(pd_ctx* ctx, const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr,
                            uint32_t n_genes, const int32_t* genome_ptr, uint32_t n_genomes, const uint32_t* jobs,
                            const int32_t* job_k, uint32_t n_jobs, uint32_t n_sample, pd_batch_tuning* best,
                            double* ms_per_job);
/* Best Hits of every job as one CSR: the rows of job j are the genes of A then
 * the genes of B (jobs in order); row_ptr n_rows+1 int64; cols int32, the
 * column's index inside the partner genome (B for rows of A, A for rows of B);
 * s uint32 sum-min.  Host or device pointers, NULL to skip. */
pd_status pd_batch_copy_hits(pd_ctx* ctx, const pd_batch* batch, int64_t* row_ptr, int32_t* cols, uint32_t* s);
/* BBH pairs of every job: job_ptr n_jobs+1 int64 offsets; pair p of job j is
 * (a[p] local in A, b[p] local in B), ascending (a, b) inside each job.  Host
 * or device pointers, NULL to skip. */
pd_status pd_batch_copy_bbh(pd_ctx* ctx, const pd_batch* batch, int64_t* job_ptr, int32_t* a, int32_t* b);
void pd_batch_free(pd_batch* batch);

/* ---------------------------------------------------------------- served index */

typedef struct pd_index pd_index;
typedef struct pd_reply pd_reply;

typedef struct {
  uint64_t ticket;
  int32_t status;             /* PD_OK, or the error that failed this request */
  uint32_t snapshot_genomes;  /* resident genomes 0 .. snapshot_genomes-1 were compared */
  uint32_t n_genes;           /* genes of the submitted genome (rows) */
  uint32_t tick_requests;     /* requests that shared this request's launches */
  uint64_t n_hits;            /* Best Hit entries */
  uint64_t n_bbh;             /* BBH pairs */
  int64_t t_submit_ns, t_start_ns, t_done_ns; /* steady-clock stamps: submitted, its tick began, answered */
} pd_reply_info;

typedef struct {
  int k;
  uint32_t n_genomes;         /* resident genomes (initial + answered requests) */
  uint64_t n_genes;
  uint32_t queued;            /* requests waiting for admission */
  uint32_t max_tick_requests; /* most requests answered by one tick */
  uint64_t device_bytes;      /* resident residues + index */
  uint64_t budget;
  uint64_t ticks;             /* launch sequences run */
  uint64_t requests_done;
} pd_index_info;

/* Served form: a pangenome index kept on the device, answering incoming
 * genomes.  The index starts from the dataset given here (offsets as in
 * pd_build_profiles; residues host or device) at a fixed k (the k rule of
 * Eq. (4) is applied by the caller, on the resident set, once).  A request
 * (pd_index_submit) is one genome: its answer holds the Best Hits (Eq. (8))
 * of each of its genes in every genome resident when it was submitted, and
 * its Bidirectional Best Hits (Eq. (9)) with those genomes; after answering,
 * the genome becomes resident (genome id = n_genomes at that moment, genes
 * appended in order).
 * The resident genomes are indexed in two levels (a base, and a delta of the
 * genomes inserted since the base was built, merged into a new base once it
 * holds a quarter of the base's windows); a request's genes are profiled
 * against each level's dictionary.
 * A worker thread of the library admits queued requests in arrival order while
 * its estimate of device memory (resident residues and index, the rebuild and
 * the tick's outputs) stays within hbm_budget bytes, and answers all admitted
 * requests with one launch sequence (continuous batching).  A request's answer
 * depends only on its genome and its snapshot, not on the requests that
 * shared its launches.  Work runs on a stream and memory pool of the index's
 * own; ctx supplies the device and receives creation errors. */
pd_status pd_index_create(pd_ctx* ctx, const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr,
                          uint32_t n_genes, const int32_t* genome_ptr, uint32_t n_genomes, int k,
                          uint64_t hbm_budget, pd_index** out);
/* Queue one genome (HOST buffers, copied before return): residues and its
 * gene_ptr (n_genes+1 int64 from 0 to n_res).  *ticket identifies the request.
 * Errors: PD_ERR_ARG (malformed), PD_ERR_ALPHABET, PD_ERR_GENE_TOO_LONG, PD_ERR_BUDGET (this
 * genome cannot fit the budget next to the resident index), PD_ERR_BUSY (the
 * index would exceed PD_MAX_GENOMES). */
pd_status pd_index_submit(pd_index* index, const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr,
                          uint32_t n_genes, uint64_t* ticket);
/* Wait up to wait_ms (negative: no limit) for a request's answer; on PD_OK
 * *out receives it (the caller frees it with pd_reply_free); PD_ERR_TIMEOUT if
 * it is not ready.  Each answer is returned once. */
pd_status pd_index_poll(pd_index* index, uint64_t ticket, int wait_ms, pd_reply** out);
pd_status pd_index_get_info(pd_index* index, pd_index_info* info);
/* Admission control (no counterpart in the paper, which has no request
 * loop).  hold != 0: the worker admits no further request -- a tick already
 * running finishes, submissions still queue; hold == 0: admission resumes,
 * and every request queued meanwhile is admitted under the budget rule above
 * (so a burst submitted while held shares its launches).  Errors: PD_ERR_ARG
 * (null index). */
pd_status pd_index_hold(pd_index* index, int hold);
/* genome_ptr of the first n_genomes resident genomes (n_genomes+1 int32, host). */
pd_status pd_index_genome_ptr(pd_index* index, uint32_t n_genomes, int32_t* genome_ptr);
/* Stops the worker (after its current tick) and frees the index; requests
 * still queued are dropped. */
void pd_index_free(pd_index* index);

pd_status pd_reply_get_info(const pd_reply* reply, pd_reply_info* info);
const char* pd_reply_error(const pd_reply* reply);
/* Answer arrays (HOST pointers, NULL to skip): row_ptr n_genes+1 int64; cols
 * n_hits int32 resident gene ids; s n_hits uint32 sum-min; bbh_a n_bbh int32
 * gene of the submitted genome; bbh_b n_bbh int32 resident gene id.  Rows and
 * pairs ascending.  Returns the request's status if it failed. */
pd_status pd_reply_copy(const pd_reply* reply, int64_t* row_ptr, int32_t* cols, uint32_t* s, int32_t* bbh_a,
                        int32_t* bbh_b);
void pd_reply_free(pd_reply* reply);

/* ---------------------------------------------------------------- no allocation */

/* Scratch of pd_best_hits_noalloc: one fixed array in device memory, held by
 * every GPU that loads this library until the process exits. */
#define PD_NOALLOC_SCRATCH_BYTES (32u << 20)
#define PD_NOALLOC_MAX_ROWS 32768u     /* genes of the query genome gi */
#define PD_NOALLOC_MAX_TARGETS 32768u  /* genes of the target genome gj */
#define PD_NOALLOC_MAX_HITS (1u << 20) /* Best Hit entries of one call */

/* The paper has no counterpart to this call: it exists for callers of this
 * library that cannot allocate device memory while they run -- a process whose
 * device memory is all owned by an external pool or memory manager, or a
 * latency-critical loop where an allocation could block or fail.
 *
 * Same result as pd_best_hits(ctx, prof, gi, gj) followed by pd_hits_copy,
 * written into caller-owned DEVICE buffers: row_ptr (|G_gi|+1 int64), cols
 * and s (capacity entries each; int32 local column, uint32 sum-min).  The
 * call allocates nothing: every temporary lives in a fixed array of
 * PD_NOALLOC_SCRATCH_BYTES declared by the library, and no per-kernel timing
 * events are recorded.  *n_hits (if not NULL) receives the number of entries.
 * Limits: |G_gi| <= PD_NOALLOC_MAX_ROWS and |G_gj| <= PD_NOALLOC_MAX_TARGETS
 * (else PD_ERR_ARG), at most PD_NOALLOC_MAX_HITS entries (else PD_ERR_BUDGET),
 * and capacity >= the entry count (else PD_ERR_ARG, *n_hits set).
 * The first call on a device looks up the array's device address (set-up,
 * once per device) and keeps it for the life of the device's primary context
 * (after cudaDeviceReset the library must be reloaded); make that first call
 * before any stream capture.  row_ptr, cols and s must be device memory of
 * ctx's device.  All
 * calls share the one array, which keeps the last call's contents: calls that
 * overlap on the GPU (other streams, other host threads, other contexts) race
 * and must be serialized by the caller.  The call synchronizes ctx's stream. */
pd_status pd_best_hits_noalloc(pd_ctx* ctx, const pd_profiles* prof, uint32_t gi, uint32_t gj, int64_t* row_ptr,
                               int32_t* cols, uint32_t* s, uint64_t capacity, uint64_t* n_hits);

#ifdef __cplusplus
}
#endif

#endif /* PD_H_ */
