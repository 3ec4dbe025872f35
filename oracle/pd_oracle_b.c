/*
 * pd_oracle_b.c -- second CPU oracle of the PanDelos-plus hot path, written
 * independently of pd_oracle.c: an inverted index walked by host threads.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite and the CPU legs of the
 * benchmark load this library.  The product path (the CUDA library) never
 * calls it and shares no code with it; it shares no code with pd_oracle.c
 * either, so that the two oracles check each other.
 *
 * Where pd_oracle.c fills the dense matrix S_ij of a genome pair (the
 * definition, "Best Hit detection phase"), this oracle follows the paper's
 * data decomposition for multicore CPUs ("Parallel implementation": a pool of
 * threads, each taking query genes in turn) and reaches the same integers by
 * another route, so that whole datasets can be checked:
 *
 *   k-mer codes           Eq. (1) and Algorithm 1: window p of a gene is the
 *       k letters g[p .. p+k-1] (there are |g|-k+1 of them, none when
 *       |g| < k), read as a number in base |Gamma| (letters numbered in the
 *       fixed order ACDEFGHIKLMNPQRSTVWY, or ACGT), first letter most
 *       significant: an injective f as Eqs. (2)-(3) require.
 *   multiplicity vectors  Algorithm 1: a gene's codes sorted, equal codes
 *       counted: (code, mult) ascending by code.
 *   inverted index        for every distinct code, the genes holding it and
 *       their multiplicities, ascending by gene.
 *   sum min               Eq. (5) numerator: for a query gene a, every
 *       posting (b, mult_b) of every code of a adds min(mult_a, mult_b) to a
 *       per-thread dense counter of b; genes b sharing no code keep 0.
 *   Best Hits             Eq. (8): per target genome, the genes b with
 *       sum min >= 1 maximising s / (La + Lb - s) (the Eq. (5) identity
 *       sum max = La + Lb - sum min; pd_oracle.c checks it on every pair it
 *       compares), compared by 64-bit cross-multiplication, every tie kept,
 *       ascending b.
 *   BBH                   Eq. (9) as read for Algorithm 3: (a, b) with
 *       genome(a) < genome(b), b a Best Hit of a in genome(b) and a a Best Hit
 *       of b in genome(a).
 *
 * Readings shared with pd_oracle.c: a candidate needs sum min >= 1; a row
 * without a candidate is empty; a gene with no window never hits and is never
 * hit; genes are compared only across genomes unless the caller lists its own
 * genome as a target (then the gene itself is still excluded).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORB_OK 0
#define ORB_ERR_ARG 1
#define ORB_ERR_ALPHABET 2
#define ORB_ERR_OOM 4

typedef struct {
  uint32_t n_genes, n_genomes;
  int k, alphabet;
  uint32_t* genome_of;   /* [G] */
  uint32_t* La;          /* [G] windows per gene */
  int32_t* genome_ptr;   /* [n+1] */
  /* multiplicity vectors, CSR over genes */
  uint64_t* mv_ptr;      /* [G+1] */
  uint64_t* mv_code;     /* [E] */
  uint32_t* mv_cnt;      /* [E] */
  uint64_t* mv_list;     /* [E] index of the entry's posting list */
  /* inverted index, CSR over distinct codes */
  uint64_t n_lists;
  uint64_t* list_ptr;    /* [D+1] */
  uint32_t* post_gene;   /* [E] ascending within a list */
  uint32_t* post_cnt;    /* [E] */
} orb_index;

typedef struct {
  uint32_t n_rows;
  int64_t* row_ptr;  /* [n_rows+1] */
  int32_t* cols;     /* global gene ids, ascending per row */
  uint32_t* s;
  uint64_t n;
} orb_hits;

static int letter_value(uint8_t c, int alphabet) {
  static const char amino[] = "ACDEFGHIKLMNPQRSTVWY";
  static const char nucleo[] = "ACGT";
  const char* t = alphabet == 4 ? nucleo : amino;
  for (int i = 0; t[i]; ++i)
    if ((uint8_t)t[i] == c) return i;
  return -1;
}

static int cmp_u64(const void* x, const void* y) {
  uint64_t a = *(const uint64_t*)x, b = *(const uint64_t*)y;
  return (a > b) - (a < b);
}

void orb_free(orb_index* X) {
  if (!X) return;
  free(X->genome_of);
  free(X->La);
  free(X->genome_ptr);
  free(X->mv_ptr);
  free(X->mv_code);
  free(X->mv_cnt);
  free(X->mv_list);
  free(X->list_ptr);
  free(X->post_gene);
  free(X->post_cnt);
  free(X);
}

/* ---------------------------------------------------------------- build */

typedef struct {
  orb_index* X;
  const uint8_t* res;
  const int64_t* gene_ptr;
  uint32_t g0, g1;
  int status;
} mv_job;

/* Multiplicity vectors of genes [g0, g1) (Algorithm 1); the entries go at
 * mv_ptr[g], which the caller has sized by La (an upper bound). */
static void* mv_worker(void* arg) {
  mv_job* J = (mv_job*)arg;
  orb_index* X = J->X;
  const int k = X->k;
  uint64_t cap = 0;
  uint64_t* tmp = NULL;
  int value[256];
  for (int c = 0; c < 256; ++c) value[c] = letter_value((uint8_t)c, X->alphabet);
  for (uint32_t g = J->g0; g < J->g1; ++g) {
    const uint8_t* s = J->res + J->gene_ptr[g];
    const uint64_t len = (uint64_t)(J->gene_ptr[g + 1] - J->gene_ptr[g]);
    const uint64_t La = len >= (uint64_t)k ? len - (uint64_t)k + 1 : 0;
    if (La > cap) {
      free(tmp);
      cap = La;
      tmp = (uint64_t*)malloc(sizeof(uint64_t) * cap);
      if (!tmp) {
        J->status = ORB_ERR_OOM;
        return NULL;
      }
    }
    for (uint64_t i = 0; i < len; ++i)
      if (value[s[i]] < 0) {
        J->status = ORB_ERR_ALPHABET;
        free(tmp);
        return NULL;
      }
    for (uint64_t p = 0; p < La; ++p) {
      uint64_t code = 0;
      for (int t = 0; t < k; ++t) code = code * (uint64_t)X->alphabet + (uint64_t)value[s[p + t]];
      tmp[p] = code;
    }
    qsort(tmp, La, sizeof(uint64_t), cmp_u64);
    uint64_t o = X->mv_ptr[g];
    for (uint64_t p = 0; p < La;) {
      uint64_t q = p;
      while (q < La && tmp[q] == tmp[p]) ++q;
      X->mv_code[o] = tmp[p];
      X->mv_cnt[o] = (uint32_t)(q - p);
      ++o;
      p = q;
    }
    X->La[g] = (uint32_t)La;
    /* entries actually used (the caller compacts with this end); a gene
     * without windows owns no slot and writes nothing */
    if (La) X->mv_list[X->mv_ptr[g]] = o;
  }
  free(tmp);
  return NULL;
}

static int run_threads(void* (*fn)(void*), void* jobs, size_t job_size, int n) {
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n);
  if (!th) return ORB_ERR_OOM;
  int started = 0;
  for (int i = 0; i < n; ++i) {
    if (pthread_create(&th[i], NULL, fn, (char*)jobs + (size_t)i * job_size) != 0) break;
    ++started;
  }
  for (int i = started; i < n; ++i) fn((char*)jobs + (size_t)i * job_size);  /* no thread: run inline */
  for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
  free(th);
  return ORB_OK;
}

/* Stable LSD radix sort of (code, entry) pairs by code, 16 bits per pass. */
static int sort_by_code(uint64_t* code, uint64_t* ent, uint64_t n, int bits) {
  uint64_t* c2 = (uint64_t*)malloc(sizeof(uint64_t) * (n ? n : 1));
  uint64_t* e2 = (uint64_t*)malloc(sizeof(uint64_t) * (n ? n : 1));
  uint64_t* cnt = (uint64_t*)malloc(sizeof(uint64_t) * 65536);
  if (!c2 || !e2 || !cnt) {
    free(c2);
    free(e2);
    free(cnt);
    return ORB_ERR_OOM;
  }
  for (int shift = 0; shift < bits; shift += 16) {
    memset(cnt, 0, sizeof(uint64_t) * 65536);
    for (uint64_t i = 0; i < n; ++i) cnt[(code[i] >> shift) & 0xFFFF]++;
    uint64_t run = 0;
    for (int d = 0; d < 65536; ++d) {
      uint64_t c = cnt[d];
      cnt[d] = run;
      run += c;
    }
    for (uint64_t i = 0; i < n; ++i) {
      uint64_t o = cnt[(code[i] >> shift) & 0xFFFF]++;
      c2[o] = code[i];
      e2[o] = ent[i];
    }
    memcpy(code, c2, sizeof(uint64_t) * n);
    memcpy(ent, e2, sizeof(uint64_t) * n);
  }
  free(c2);
  free(e2);
  free(cnt);
  return ORB_OK;
}

orb_index* orb_build(const uint8_t* res, uint64_t n_res, const int64_t* gene_ptr, uint32_t n_genes,
                     const int32_t* genome_ptr, uint32_t n_genomes, int k, int alphabet, int n_threads,
                     int* status) {
  *status = ORB_ERR_ARG;
  if (k < 1 || (alphabet != 20 && alphabet != 4) || n_genomes < 1 || n_threads < 1) return NULL;
  if (gene_ptr[0] != 0 || (uint64_t)gene_ptr[n_genes] != n_res) return NULL;
  if (genome_ptr[0] != 0 || (uint32_t)genome_ptr[n_genomes] != n_genes) return NULL;
  /* codes must fit 64 bits: alphabet^k < 2^64 */
  {
    unsigned __int128 p = 1;
    for (int t = 0; t < k; ++t) p *= (unsigned)alphabet;
    if (p > (unsigned __int128)UINT64_MAX) return NULL;
  }
  *status = ORB_ERR_OOM;
  orb_index* X = (orb_index*)calloc(1, sizeof(orb_index));
  if (!X) return NULL;
  X->n_genes = n_genes;
  X->n_genomes = n_genomes;
  X->k = k;
  X->alphabet = alphabet;
  X->genome_of = (uint32_t*)malloc(sizeof(uint32_t) * (n_genes ? n_genes : 1));
  X->La = (uint32_t*)calloc(n_genes ? n_genes : 1, sizeof(uint32_t));
  X->genome_ptr = (int32_t*)malloc(sizeof(int32_t) * (n_genomes + 1));
  X->mv_ptr = (uint64_t*)malloc(sizeof(uint64_t) * (n_genes + 1));
  if (!X->genome_of || !X->La || !X->genome_ptr || !X->mv_ptr) goto fail;
  memcpy(X->genome_ptr, genome_ptr, sizeof(int32_t) * (n_genomes + 1));
  for (uint32_t i = 0; i < n_genomes; ++i) {
    if (genome_ptr[i + 1] < genome_ptr[i]) {
      *status = ORB_ERR_ARG;
      goto fail;
    }
    for (int32_t g = genome_ptr[i]; g < genome_ptr[i + 1]; ++g) X->genome_of[g] = i;
  }
  /* upper bound of each gene's entries: its windows */
  uint64_t W = 0;
  X->mv_ptr[0] = 0;
  for (uint32_t g = 0; g < n_genes; ++g) {
    if (gene_ptr[g + 1] < gene_ptr[g]) {
      *status = ORB_ERR_ARG;
      goto fail;
    }
    const uint64_t len = (uint64_t)(gene_ptr[g + 1] - gene_ptr[g]);
    W += len >= (uint64_t)k ? len - (uint64_t)k + 1 : 0;
    X->mv_ptr[g + 1] = W;
  }
  X->mv_code = (uint64_t*)malloc(sizeof(uint64_t) * (W ? W : 1));
  X->mv_cnt = (uint32_t*)malloc(sizeof(uint32_t) * (W ? W : 1));
  X->mv_list = (uint64_t*)malloc(sizeof(uint64_t) * (W ? W : 1));
  if (!X->mv_code || !X->mv_cnt || !X->mv_list) goto fail;
  {
    mv_job* jobs = (mv_job*)calloc((size_t)n_threads, sizeof(mv_job));
    if (!jobs) goto fail;
    for (int t = 0; t < n_threads; ++t) {
      jobs[t].X = X;
      jobs[t].res = res;
      jobs[t].gene_ptr = gene_ptr;
      jobs[t].g0 = (uint32_t)((uint64_t)n_genes * (uint64_t)t / (uint64_t)n_threads);
      jobs[t].g1 = (uint32_t)((uint64_t)n_genes * (uint64_t)(t + 1) / (uint64_t)n_threads);
    }
    int st = run_threads(mv_worker, jobs, sizeof(mv_job), n_threads);
    for (int t = 0; t < n_threads && st == ORB_OK; ++t) st = jobs[t].status;
    free(jobs);
    if (st != ORB_OK) {
      *status = st;
      goto fail;
    }
  }
  /* compact the vectors (each gene used mv_list[mv_ptr[g]] - mv_ptr[g] slots) */
  {
    uint64_t o = 0;
    for (uint32_t g = 0; g < n_genes; ++g) {
      const uint64_t b = X->mv_ptr[g], e = X->La[g] ? X->mv_list[b] : b;
      memmove(X->mv_code + o, X->mv_code + b, sizeof(uint64_t) * (e - b));
      memmove(X->mv_cnt + o, X->mv_cnt + b, sizeof(uint32_t) * (e - b));
      X->mv_ptr[g] = o;
      o += e - b;
    }
    X->mv_ptr[n_genes] = o;
  }
  const uint64_t E = X->mv_ptr[n_genes];
  /* inverted index: entries sorted by code, stably (so by gene inside a code) */
  {
    uint64_t* code = (uint64_t*)malloc(sizeof(uint64_t) * (E ? E : 1));
    uint64_t* ent = (uint64_t*)malloc(sizeof(uint64_t) * (E ? E : 1));
    if (!code || !ent) {
      free(code);
      free(ent);
      goto fail;
    }
    memcpy(code, X->mv_code, sizeof(uint64_t) * E);
    for (uint64_t e = 0; e < E; ++e) ent[e] = e;
    uint64_t maxc = 0;
    for (uint64_t e = 0; e < E; ++e)
      if (code[e] > maxc) maxc = code[e];
    int bits = 0;
    while (bits < 64 && (maxc >> bits) != 0) bits += 16;
    if (sort_by_code(code, ent, E, bits) != ORB_OK) {
      free(code);
      free(ent);
      goto fail;
    }
    uint64_t D = 0;
    for (uint64_t i = 0; i < E; ++i)
      if (i == 0 || code[i] != code[i - 1]) ++D;
    X->n_lists = D;
    X->list_ptr = (uint64_t*)malloc(sizeof(uint64_t) * (D + 1));
    X->post_gene = (uint32_t*)malloc(sizeof(uint32_t) * (E ? E : 1));
    X->post_cnt = (uint32_t*)malloc(sizeof(uint32_t) * (E ? E : 1));
    uint32_t* gene_of_entry = (uint32_t*)malloc(sizeof(uint32_t) * (E ? E : 1));
    if (!X->list_ptr || !X->post_gene || !X->post_cnt || !gene_of_entry) {
      free(code);
      free(ent);
      free(gene_of_entry);
      goto fail;
    }
    for (uint32_t g = 0; g < n_genes; ++g)
      for (uint64_t e = X->mv_ptr[g]; e < X->mv_ptr[g + 1]; ++e) gene_of_entry[e] = g;
    uint64_t d = 0;
    for (uint64_t i = 0; i < E; ++i) {
      if (i == 0 || code[i] != code[i - 1]) X->list_ptr[d++] = i;
      X->post_gene[i] = gene_of_entry[ent[i]];
      X->post_cnt[i] = X->mv_cnt[ent[i]];
      X->mv_list[ent[i]] = d - 1;
    }
    X->list_ptr[D] = E;
    free(code);
    free(ent);
    free(gene_of_entry);
  }
  *status = ORB_OK;
  return X;
fail:
  orb_free(X);
  return NULL;
}

uint64_t orb_n_entries(const orb_index* X) { return X->mv_ptr[X->n_genes]; }
uint64_t orb_n_lists(const orb_index* X) { return X->n_lists; }
uint32_t orb_La(const orb_index* X, uint32_t g) { return X->La[g]; }

/* ---------------------------------------------------------------- Best Hits */

typedef struct {
  const orb_index* X;
  const uint32_t* queries;
  uint32_t n_q;
  const uint8_t* target_genome;  /* [n_genomes]: 1 = target (the query's own genome included if set) */
  int own_genome;                /* 1: each query also targets its own genome (itself excluded) */
  volatile uint32_t* next;       /* shared work counter */
  pthread_mutex_t* mu;
  /* per query: its row (malloc'ed), filled by whichever thread took it */
  uint32_t** row_cols;
  uint32_t** row_s;
  uint32_t* row_len;
  int status;
} bh_job;

static int ratio_cmp(uint32_t s1, uint32_t d1, uint32_t s2, uint32_t d2) {
  const uint64_t x = (uint64_t)s1 * (uint64_t)d2, y = (uint64_t)s2 * (uint64_t)d1;
  return (x > y) - (x < y);
}

static int cmp_u32(const void* x, const void* y) {
  uint32_t a = *(const uint32_t*)x, b = *(const uint32_t*)y;
  return (a > b) - (a < b);
}

static void* bh_worker(void* arg) {
  bh_job* J = (bh_job*)arg;
  const orb_index* X = J->X;
  const uint32_t G = X->n_genes;
  uint32_t* acc = (uint32_t*)calloc(G ? G : 1, sizeof(uint32_t));
  uint32_t* touched = (uint32_t*)malloc(sizeof(uint32_t) * (G ? G : 1));
  uint32_t* best_s = (uint32_t*)calloc(X->n_genomes, sizeof(uint32_t));
  uint32_t* best_d = (uint32_t*)calloc(X->n_genomes, sizeof(uint32_t));
  uint32_t* hit = (uint32_t*)malloc(sizeof(uint32_t) * (G ? G : 1));
  if (!acc || !touched || !best_s || !best_d || !hit) {
    J->status = ORB_ERR_OOM;
    goto out;
  }
  for (;;) {
    uint32_t q;
    pthread_mutex_lock(J->mu);
    q = *J->next;
    if (q < J->n_q) *J->next = q + 1;
    pthread_mutex_unlock(J->mu);
    if (q >= J->n_q) break;
    const uint32_t a = J->queries[q];
    const uint32_t ga = X->genome_of[a];
    uint32_t n_t = 0;
    /* sum min of a with every gene sharing a code (Eq. (5) numerator) */
    for (uint64_t e = X->mv_ptr[a]; e < X->mv_ptr[a + 1]; ++e) {
      const uint32_t ca = X->mv_cnt[e];
      const uint64_t l = X->mv_list[e];
      for (uint64_t p = X->list_ptr[l]; p < X->list_ptr[l + 1]; ++p) {
        const uint32_t b = X->post_gene[p];
        const uint32_t gb = X->genome_of[b];
        if (b == a) continue;
        if (gb == ga ? !J->own_genome : !J->target_genome[gb]) continue;
        const uint32_t cb = X->post_cnt[p];
        if (acc[b] == 0) touched[n_t++] = b;
        acc[b] += ca < cb ? ca : cb;
      }
    }
    /* per target genome: the largest s / (La + Lb - s) (Eq. (8)) */
    for (uint32_t t = 0; t < n_t; ++t) {
      const uint32_t b = touched[t], gb = X->genome_of[b];
      const uint32_t s = acc[b], den = X->La[a] + X->La[b] - s;
      if (best_s[gb] == 0 || ratio_cmp(s, den, best_s[gb], best_d[gb]) > 0) {
        best_s[gb] = s;
        best_d[gb] = den;
      }
    }
    uint32_t n_hit = 0;
    for (uint32_t t = 0; t < n_t; ++t) {
      const uint32_t b = touched[t], gb = X->genome_of[b];
      const uint32_t s = acc[b], den = X->La[a] + X->La[b] - s;
      if (ratio_cmp(s, den, best_s[gb], best_d[gb]) == 0) hit[n_hit++] = b;
    }
    qsort(hit, n_hit, sizeof(uint32_t), cmp_u32);
    uint32_t* rc = (uint32_t*)malloc(sizeof(uint32_t) * (n_hit ? n_hit : 1));
    uint32_t* rs = (uint32_t*)malloc(sizeof(uint32_t) * (n_hit ? n_hit : 1));
    if (!rc || !rs) {
      free(rc);
      free(rs);
      J->status = ORB_ERR_OOM;
      goto out;
    }
    for (uint32_t h = 0; h < n_hit; ++h) {
      rc[h] = hit[h];
      rs[h] = acc[hit[h]];
    }
    J->row_cols[q] = rc;
    J->row_s[q] = rs;
    J->row_len[q] = n_hit;
    for (uint32_t t = 0; t < n_t; ++t) {
      const uint32_t b = touched[t];
      best_s[X->genome_of[b]] = 0;
      best_d[X->genome_of[b]] = 0;
      acc[b] = 0;
    }
  }
out:
  free(acc);
  free(touched);
  free(best_s);
  free(best_d);
  free(hit);
  return NULL;
}

void orb_hits_free(orb_hits* H) {
  if (!H) return;
  free(H->row_ptr);
  free(H->cols);
  free(H->s);
  free(H);
}

/* Best Hits of the listed query genes towards the target genomes (mask, one
 * byte per genome; NULL = every genome but the query's own), own_genome = 1
 * adds the query's own genome (the gene itself excluded). */
orb_hits* orb_best_hits(const orb_index* X, const uint32_t* queries, uint32_t n_q, const uint8_t* target_genome,
                        int own_genome, int n_threads, int* status) {
  *status = ORB_ERR_ARG;
  if (!X || n_threads < 1) return NULL;
  for (uint32_t q = 0; q < n_q; ++q)
    if (queries[q] >= X->n_genes) return NULL;
  *status = ORB_ERR_OOM;
  uint8_t* mask = (uint8_t*)malloc(X->n_genomes);
  orb_hits* H = (orb_hits*)calloc(1, sizeof(orb_hits));
  uint32_t** rc = (uint32_t**)calloc(n_q ? n_q : 1, sizeof(uint32_t*));
  uint32_t** rs = (uint32_t**)calloc(n_q ? n_q : 1, sizeof(uint32_t*));
  uint32_t* rl = (uint32_t*)calloc(n_q ? n_q : 1, sizeof(uint32_t));
  bh_job* jobs = (bh_job*)calloc((size_t)n_threads, sizeof(bh_job));
  if (!mask || !H || !rc || !rs || !rl || !jobs) goto fail;
  for (uint32_t g = 0; g < X->n_genomes; ++g) mask[g] = target_genome ? (target_genome[g] != 0) : 1;
  {
    volatile uint32_t next = 0;
    pthread_mutex_t mu = PTHREAD_MUTEX_INITIALIZER;
    for (int t = 0; t < n_threads; ++t) {
      jobs[t].X = X;
      jobs[t].queries = queries;
      jobs[t].n_q = n_q;
      jobs[t].target_genome = mask;
      jobs[t].own_genome = own_genome;
      jobs[t].next = &next;
      jobs[t].mu = &mu;
      jobs[t].row_cols = rc;
      jobs[t].row_s = rs;
      jobs[t].row_len = rl;
    }
    int st = run_threads(bh_worker, jobs, sizeof(bh_job), n_threads);
    for (int t = 0; t < n_threads && st == ORB_OK; ++t) st = jobs[t].status;
    if (st != ORB_OK) goto fail;
  }
  H->n_rows = n_q;
  H->row_ptr = (int64_t*)malloc(sizeof(int64_t) * (n_q + 1));
  if (!H->row_ptr) goto fail;
  H->row_ptr[0] = 0;
  for (uint32_t q = 0; q < n_q; ++q) H->row_ptr[q + 1] = H->row_ptr[q] + rl[q];
  H->n = (uint64_t)H->row_ptr[n_q];
  H->cols = (int32_t*)malloc(sizeof(int32_t) * (H->n ? H->n : 1));
  H->s = (uint32_t*)malloc(sizeof(uint32_t) * (H->n ? H->n : 1));
  if (!H->cols || !H->s) goto fail;
  for (uint32_t q = 0; q < n_q; ++q) {
    for (uint32_t h = 0; h < rl[q]; ++h) {
      H->cols[H->row_ptr[q] + h] = (int32_t)rc[q][h];
      H->s[H->row_ptr[q] + h] = rs[q][h];
    }
  }
  for (uint32_t q = 0; q < n_q; ++q) {
    free(rc[q]);
    free(rs[q]);
  }
  free(rc);
  free(rs);
  free(rl);
  free(jobs);
  free(mask);
  *status = ORB_OK;
  return H;
fail:
  if (rc)
    for (uint32_t q = 0; q < n_q; ++q) free(rc[q]);
  if (rs)
    for (uint32_t q = 0; q < n_q; ++q) free(rs[q]);
  free(rc);
  free(rs);
  free(rl);
  free(jobs);
  free(mask);
  orb_hits_free(H);
  return NULL;
}

uint32_t orb_hits_rows(const orb_hits* H) { return H->n_rows; }
uint64_t orb_hits_count(const orb_hits* H) { return H->n; }

void orb_hits_get(const orb_hits* H, int64_t* row_ptr, int32_t* cols, uint32_t* s) {
  memcpy(row_ptr, H->row_ptr, sizeof(int64_t) * (H->n_rows + 1));
  if (H->n) {
    memcpy(cols, H->cols, sizeof(int32_t) * H->n);
    memcpy(s, H->s, sizeof(uint32_t) * H->n);
  }
}

/* ---------------------------------------------------------------- BBH */

static int row_has(const orb_hits* H, uint32_t row, int32_t x) {
  int64_t lo = H->row_ptr[row], hi = H->row_ptr[row + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (H->cols[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo < H->row_ptr[row + 1] && H->cols[lo] == x;
}

/* From Best Hits of every gene (queries 0..G-1 in order, every other genome
 * a target): the BBH pairs (a, b), genome(a) < genome(b), ascending.  Writes
 * at most cap pairs and returns the count (pass cap 0 to size). */
uint64_t orb_bbh(const orb_index* X, const orb_hits* H, int32_t* a_out, int32_t* b_out, uint64_t cap) {
  uint64_t n = 0;
  if (H->n_rows != X->n_genes) return 0;
  for (uint32_t a = 0; a < X->n_genes; ++a) {
    for (int64_t p = H->row_ptr[a]; p < H->row_ptr[a + 1]; ++p) {
      const uint32_t b = (uint32_t)H->cols[p];
      if (X->genome_of[b] <= X->genome_of[a]) continue;
      if (!row_has(H, b, (int32_t)a)) continue;
      if (n < cap) {
        a_out[n] = (int32_t)a;
        b_out[n] = (int32_t)b;
      }
      ++n;
    }
  }
  return n;
}
