/*
 * pd_oracle.c -- plain, slow, CPU reference of the PanDelos-plus hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library) never calls it and shares no code with it.
 *
 * What it computes, each step written out from its definition:
 *
 *   k-mer dictionary and multiplicities   Eqs. (1)-(3), "Basic notions":
 *       the k-mers of a gene are its |g|-k+1 windows of exactly k letters
 *       (Algorithm 1 slides p over 1..|g|-k+1 and reads g[p..p+k-1]); a gene
 *       shorter than k has none.  mult_g(w) counts the windows equal to w.
 *   multiplicity vector (MV)              Algorithm 1, "Multiplicity vector
 *       building phase": the distinct k-mers of a gene with their counts, in
 *       ascending order of an injective id f.  Here f is the lexicographic
 *       order of the k-mer strings (bytes compared with memcmp), and the
 *       k-mers are kept as strings -- no numeric encoding at all.
 *   generalized Jaccard                   Eq. (5):
 *       J = sum_{w in D(a) & D(b)} min(mult) / sum_{w in D(a) | D(b)} max(mult).
 *       Both sums are taken literally, by walking the two sorted MVs
 *       together; the identity  sum max = La + Lb - sum min  (La = number of
 *       windows of a) is checked on every pair and any mismatch is reported.
 *   similarity matrix S_ij                "Best Hit detection phase": the dense
 *       |G_i| x |G_j| matrix of (sum min, sum max) values.
 *   Best Hits                             Eq. (8), Algorithm 2: for each row,
 *       the set of all columns that attain the row maximum of J.
 *   Bidirectional Best Hits               Eq. (9), Algorithm 3: for each
 *       relevant column k and each row l with k in A_ij[l], keep (l, k) when
 *       S[l,k] equals the column maximum and l is in A_ji[k].
 *
 * Readings of points the paper leaves open (kept identical on every side):
 *   - ratios are compared exactly, by 64-bit cross-multiplication
 *     (s1 * den2 versus s2 * den1); no floating point is used anywhere;
 *   - a pair is a candidate only if sum min >= 1 ("minimum overlap between
 *     the k-dictionaries", "PanDelos methodology"); a row without a candidate
 *     has an empty Best Hit set (Eq. (8) alone would make every column a Best
 *     Hit of a zero row, and J is 0/0 when both genes have no window);
 *   - Eq. (9) names BH(g_jk, G_j); the relation intended (and used by
 *     Algorithm 3) is BH(g_jk, G_i);
 *   - the alphabet is the 20 upper-case amino-acid letters; any other byte
 *     is rejected.
 *   - k selection (Eq. (4)) reads sum |G_i| as the total number of residues
 *     and takes the smallest integer k with |Gamma|^k >= that total.
 *     PARITY UNPINNED: the paper prints no k for any dataset; k is an
 *     explicit input everywhere else, so no other result depends on it.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_ALPHABET 2
#define ORC_ERR_IDENTITY 3
#define ORC_ERR_OOM 4

static const char kAmino[] = "ACDEFGHIKLMNPQRSTVWY";
static const char kNucleotide[] = "ACGT";

/* "nucleotide or amino acid" alphabets (Basic notions): 20 upper-case amino
 * acids, or the 4 upper-case nucleotides. */
static int valid_letter(uint8_t c, int alphabet) {
  const char* letters = alphabet == 4 ? kNucleotide : kAmino;
  for (int i = 0; letters[i]; ++i)
    if ((uint8_t)letters[i] == c) return 1;
  return 0;
}

/* Eq. (4), read as: smallest k >= 1 with alphabet^k >= total (parity unpinned). */
int orc_choose_k(uint64_t total, int alphabet) {
  if (alphabet < 2) return -1;
  int k = 1;
  unsigned __int128 p = (unsigned __int128)alphabet;
  while (p < total) {
    p *= (unsigned)alphabet;
    ++k;
  }
  return k;
}

/* ------------------------------------------------------------------------ */
/* Multiplicity vectors (Algorithm 1)                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
  const uint8_t* res; /* the gene's letters */
  uint32_t len;       /* |g| */
  uint32_t La;        /* number of windows: |g|-k+1, or 0 when |g| < k */
  uint32_t n;         /* number of distinct k-mers */
  uint32_t* start;    /* start offset (in the gene) of one copy of each k-mer */
  uint32_t* cnt;      /* its multiplicity */
} orc_mv;

typedef struct {
  int k;
  uint32_t n_genes;
  uint8_t* res; /* private copy of all residues */
  orc_mv* mv;
} orc_profiles;

static int g_k_for_sort; /* used only by the qsort comparator below */
static const uint8_t* g_res_for_sort;
static pthread_mutex_t g_sort_lock = PTHREAD_MUTEX_INITIALIZER;

static int cmp_window(const void* x, const void* y) {
  uint32_t a = *(const uint32_t*)x, b = *(const uint32_t*)y;
  int c = memcmp(g_res_for_sort + a, g_res_for_sort + b, (size_t)g_k_for_sort);
  if (c) return c;
  return (a > b) - (a < b);
}

/* Build the MV of one gene: sort its windows as strings, then count runs. */
static int build_mv(orc_mv* m, const uint8_t* res, uint32_t len, int k) {
  m->res = res;
  m->len = len;
  m->La = (len >= (uint32_t)k) ? len - (uint32_t)k + 1u : 0u;
  m->n = 0;
  m->start = NULL;
  m->cnt = NULL;
  if (m->La == 0) return ORC_OK;
  uint32_t* pos = (uint32_t*)malloc(sizeof(uint32_t) * m->La);
  m->start = (uint32_t*)malloc(sizeof(uint32_t) * m->La);
  m->cnt = (uint32_t*)malloc(sizeof(uint32_t) * m->La);
  if (!pos || !m->start || !m->cnt) {
    free(pos);
    return ORC_ERR_OOM;
  }
  for (uint32_t p = 0; p < m->La; ++p) pos[p] = p;
  pthread_mutex_lock(&g_sort_lock);
  g_k_for_sort = k;
  g_res_for_sort = res;
  qsort(pos, m->La, sizeof(uint32_t), cmp_window);
  pthread_mutex_unlock(&g_sort_lock);
  for (uint32_t p = 0; p < m->La; ++p) {
    if (m->n > 0 && memcmp(res + m->start[m->n - 1], res + pos[p], (size_t)k) == 0) {
      m->cnt[m->n - 1] += 1;
    } else {
      m->start[m->n] = pos[p];
      m->cnt[m->n] = 1;
      m->n += 1;
    }
  }
  free(pos);
  return ORC_OK;
}

void orc_free(orc_profiles* P) {
  if (!P) return;
  if (P->mv) {
    for (uint32_t g = 0; g < P->n_genes; ++g) {
      free(P->mv[g].start);
      free(P->mv[g].cnt);
    }
  }
  free(P->mv);
  free(P->res);
  free(P);
}

/* Build the MVs of all genes over an alphabet of 20 (amino acids) or 4
 * (nucleotides) letters.  *status receives an ORC_* code. */
orc_profiles* orc_build_alphabet(const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr,
                                 uint32_t n_genes, int k, int alphabet, int* status) {
  *status = ORC_ERR_ARG;
  if (k < 1 || (alphabet != 20 && alphabet != 4)) return NULL;
  if (!gene_ptr || gene_ptr[0] != 0 || (uint64_t)gene_ptr[n_genes] != n_res) return NULL;
  for (uint32_t g = 0; g < n_genes; ++g)
    if (gene_ptr[g + 1] < gene_ptr[g]) return NULL;
  for (uint64_t i = 0; i < n_res; ++i)
    if (!valid_letter(residues[i], alphabet)) {
      *status = ORC_ERR_ALPHABET;
      return NULL;
    }
  orc_profiles* P = (orc_profiles*)calloc(1, sizeof(orc_profiles));
  if (!P) {
    *status = ORC_ERR_OOM;
    return NULL;
  }
  P->k = k;
  P->n_genes = n_genes;
  P->res = (uint8_t*)malloc(n_res ? n_res : 1);
  P->mv = (orc_mv*)calloc(n_genes ? n_genes : 1, sizeof(orc_mv));
  if (!P->res || !P->mv) {
    orc_free(P);
    *status = ORC_ERR_OOM;
    return NULL;
  }
  if (n_res) memcpy(P->res, residues, n_res);
  for (uint32_t g = 0; g < n_genes; ++g) {
    int st = build_mv(&P->mv[g], P->res + gene_ptr[g], (uint32_t)(gene_ptr[g + 1] - gene_ptr[g]), k);
    if (st != ORC_OK) {
      orc_free(P);
      *status = st;
      return NULL;
    }
  }
  *status = ORC_OK;
  return P;
}

orc_profiles* orc_build(const uint8_t* residues, uint64_t n_res, const int64_t* gene_ptr, uint32_t n_genes, int k,
                        int* status) {
  return orc_build_alphabet(residues, n_res, gene_ptr, n_genes, k, 20, status);
}

uint32_t orc_mv_len(const orc_profiles* P, uint32_t g) { return P->mv[g].n; }
uint32_t orc_La(const orc_profiles* P, uint32_t g) { return P->mv[g].La; }

/* Copy out the MV of gene g: k-mer strings (n*k bytes) and counts. */
void orc_mv_get(const orc_profiles* P, uint32_t g, uint8_t* kmers, uint32_t* counts) {
  const orc_mv* m = &P->mv[g];
  for (uint32_t e = 0; e < m->n; ++e) {
    if (kmers) memcpy(kmers + (size_t)e * (size_t)P->k, m->res + m->start[e], (size_t)P->k);
    if (counts) counts[e] = m->cnt[e];
  }
}

/* ------------------------------------------------------------------------ */
/* Eq. (5): numerator and denominator of the generalized Jaccard           */
/* ------------------------------------------------------------------------ */

/* sum over the intersection of min(mult), and over the union of max(mult),
 * walking both sorted MVs together.  Returns ORC_ERR_IDENTITY if the union
 * sum differs from La + Lb - (intersection sum). */
static int pair_sums(const orc_mv* a, const orc_mv* b, int k, uint32_t* s_min, uint32_t* s_max) {
  uint32_t i = 0, j = 0;
  uint64_t smin = 0, smax = 0;
  while (i < a->n && j < b->n) {
    int c = memcmp(a->res + a->start[i], b->res + b->start[j], (size_t)k);
    if (c == 0) { /* w in D(a) and D(b) */
      uint32_t ca = a->cnt[i], cb = b->cnt[j];
      smin += (ca < cb) ? ca : cb;
      smax += (ca > cb) ? ca : cb;
      ++i;
      ++j;
    } else if (c < 0) { /* w only in D(a): max = mult_a(w) */
      smax += a->cnt[i];
      ++i;
    } else { /* w only in D(b) */
      smax += b->cnt[j];
      ++j;
    }
  }
  for (; i < a->n; ++i) smax += a->cnt[i];
  for (; j < b->n; ++j) smax += b->cnt[j];
  *s_min = (uint32_t)smin;
  *s_max = (uint32_t)smax;
  if (smax != (uint64_t)a->La + (uint64_t)b->La - smin) return ORC_ERR_IDENTITY;
  return ORC_OK;
}

int orc_summin(const orc_profiles* P, uint32_t a, uint32_t b, uint32_t* s_min, uint32_t* s_max) {
  if (a >= P->n_genes || b >= P->n_genes) return ORC_ERR_ARG;
  return pair_sums(&P->mv[a], &P->mv[b], P->k, s_min, s_max);
}

/* Eq. (7) numerators: the sum of mult_a(w) (and of mult_b(w)) over the
 * k-mers w in both dictionaries, by the same walk over the two sorted MVs. */
int orc_directional(const orc_profiles* P, uint32_t a, uint32_t b, uint32_t* pa, uint32_t* pb) {
  if (a >= P->n_genes || b >= P->n_genes) return ORC_ERR_ARG;
  const orc_mv* x = &P->mv[a];
  const orc_mv* y = &P->mv[b];
  uint32_t i = 0, j = 0;
  uint64_t sa = 0, sb = 0;
  while (i < x->n && j < y->n) {
    int c = memcmp(x->res + x->start[i], y->res + y->start[j], (size_t)P->k);
    if (c == 0) {
      sa += x->cnt[i];
      sb += y->cnt[j];
      ++i;
      ++j;
    } else if (c < 0) {
      ++i;
    } else {
      ++j;
    }
  }
  *pa = (uint32_t)sa;
  *pb = (uint32_t)sb;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* One genome pair: S_ij, A_ij (rows), A_ji (columns), BBH                  */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint32_t n_rows, n_cols;
  uint32_t* S;    /* n_rows*n_cols: sum min */
  uint32_t* Den;  /* n_rows*n_cols: sum max (the Eq. (5) denominator) */
  int64_t* row_ptr; /* A_ij as CSR over rows */
  int32_t* row_col;
  uint32_t* row_best_s; /* best (s, den) per row, 0/0 when the row is empty */
  uint32_t* row_best_den;
  int64_t* col_ptr; /* A_ji as CSR over columns */
  int32_t* col_row;
  uint32_t* col_best_s;
  uint32_t* col_best_den;
  uint64_t n_bbh;
  int32_t* bbh_a;
  int32_t* bbh_b;
  int status;
} orc_pair;

typedef struct {
  const orc_profiles* P;
  orc_pair* R;
  uint32_t g0_i, g0_j; /* first gene of each genome */
  uint32_t row_begin, row_end;
  int status;
} row_task;

static void* row_worker(void* arg) {
  row_task* t = (row_task*)arg;
  const orc_pair* R = t->R;
  t->status = ORC_OK;
  for (uint32_t l = t->row_begin; l < t->row_end; ++l)
    for (uint32_t c = 0; c < R->n_cols; ++c) {
      uint32_t s, d;
      int st = pair_sums(&t->P->mv[t->g0_i + l], &t->P->mv[t->g0_j + c], t->P->k, &s, &d);
      if (st != ORC_OK) t->status = st;
      R->S[(size_t)l * R->n_cols + c] = s;
      R->Den[(size_t)l * R->n_cols + c] = d;
    }
  return NULL;
}

/* x = s1/d1 compared with y = s2/d2 by cross-multiplication: -1, 0, +1 */
static int cmp_ratio(uint32_t s1, uint32_t d1, uint32_t s2, uint32_t d2) {
  uint64_t l = (uint64_t)s1 * (uint64_t)d2, r = (uint64_t)s2 * (uint64_t)d1;
  return (l > r) - (l < r);
}

/* Best Hit sets (Eq. (8)) of every line of a matrix, where line x holds the
 * values at idx(x, y) for y = 0..n_y-1.  Candidates need s >= 1.  Ties are all
 * kept, in ascending y. */
static int best_hits(const uint32_t* S, const uint32_t* D, uint32_t n_x, uint32_t n_y, int by_row,
                     int64_t** ptr_out, int32_t** idx_out, uint32_t** best_s, uint32_t** best_d) {
  int64_t* ptr = (int64_t*)calloc((size_t)n_x + 1, sizeof(int64_t));
  uint32_t* bs = (uint32_t*)calloc(n_x ? n_x : 1, sizeof(uint32_t));
  uint32_t* bd = (uint32_t*)calloc(n_x ? n_x : 1, sizeof(uint32_t));
  if (!ptr || !bs || !bd) return ORC_ERR_OOM;
  /* pass 1: the maximum of each line, and how many entries attain it */
  for (uint32_t x = 0; x < n_x; ++x) {
    uint32_t ms = 0, md = 0;
    int64_t ties = 0;
    for (uint32_t y = 0; y < n_y; ++y) {
      size_t at = by_row ? (size_t)x * n_y + y : (size_t)y * n_x + x;
      uint32_t s = S[at], d = D[at];
      if (s == 0) continue; /* not a candidate */
      if (ms == 0 || cmp_ratio(s, d, ms, md) > 0) {
        ms = s;
        md = d;
        ties = 1;
      } else if (cmp_ratio(s, d, ms, md) == 0) {
        ties += 1;
      }
    }
    bs[x] = ms;
    bd[x] = md;
    ptr[x + 1] = ptr[x] + ties;
  }
  int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ptr[n_x] ? ptr[n_x] : 1));
  if (!idx) return ORC_ERR_OOM;
  /* pass 2: list the entries that attain the maximum, in ascending order */
  for (uint32_t x = 0; x < n_x; ++x) {
    int64_t o = ptr[x];
    if (bs[x] == 0) continue;
    for (uint32_t y = 0; y < n_y; ++y) {
      size_t at = by_row ? (size_t)x * n_y + y : (size_t)y * n_x + x;
      if (S[at] != 0 && cmp_ratio(S[at], D[at], bs[x], bd[x]) == 0) idx[o++] = (int32_t)y;
    }
  }
  *ptr_out = ptr;
  *idx_out = idx;
  *best_s = bs;
  *best_d = bd;
  return ORC_OK;
}

static int contains(const int32_t* v, int64_t lo, int64_t hi, int32_t x) {
  for (int64_t t = lo; t < hi; ++t)
    if (v[t] == x) return 1;
  return 0;
}

void orc_pair_free(orc_pair* R) {
  if (!R) return;
  free(R->S);
  free(R->Den);
  free(R->row_ptr);
  free(R->row_col);
  free(R->row_best_s);
  free(R->row_best_den);
  free(R->col_ptr);
  free(R->col_row);
  free(R->col_best_s);
  free(R->col_best_den);
  free(R->bbh_a);
  free(R->bbh_b);
  free(R);
}

/* Compare genome gi (rows) with genome gj (columns).  genome_ptr holds gene
 * offsets per genome.  n_threads > 1 splits the rows of S over host threads. */
orc_pair* orc_pair_run(const orc_profiles* P, const int32_t* genome_ptr, uint32_t gi, uint32_t gj,
                       int n_threads) {
  orc_pair* R = (orc_pair*)calloc(1, sizeof(orc_pair));
  if (!R) return NULL;
  uint32_t g0_i = (uint32_t)genome_ptr[gi], g0_j = (uint32_t)genome_ptr[gj];
  R->n_rows = (uint32_t)(genome_ptr[gi + 1] - genome_ptr[gi]);
  R->n_cols = (uint32_t)(genome_ptr[gj + 1] - genome_ptr[gj]);
  size_t cells = (size_t)R->n_rows * R->n_cols;
  R->S = (uint32_t*)malloc(sizeof(uint32_t) * (cells ? cells : 1));
  R->Den = (uint32_t*)malloc(sizeof(uint32_t) * (cells ? cells : 1));
  if (!R->S || !R->Den) {
    R->status = ORC_ERR_OOM;
    return R;
  }
  /* Algorithm 2, first half: every cell of S_ij. */
  if (n_threads < 1) n_threads = 1;
  if ((uint32_t)n_threads > R->n_rows) n_threads = R->n_rows ? (int)R->n_rows : 1;
  row_task* tasks = (row_task*)calloc((size_t)n_threads, sizeof(row_task));
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  for (int t = 0; t < n_threads; ++t) {
    tasks[t].P = P;
    tasks[t].R = R;
    tasks[t].g0_i = g0_i;
    tasks[t].g0_j = g0_j;
    tasks[t].row_begin = (uint32_t)(((uint64_t)R->n_rows * t) / n_threads);
    tasks[t].row_end = (uint32_t)(((uint64_t)R->n_rows * (t + 1)) / n_threads);
  }
  for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, row_worker, &tasks[t]);
  row_worker(&tasks[0]);
  for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
  for (int t = 0; t < n_threads; ++t)
    if (tasks[t].status != ORC_OK) R->status = tasks[t].status;
  free(tasks);
  free(th);
  if (R->status != ORC_OK) return R;

  /* Algorithm 2, second half: A_ij, the Best Hits of every row. */
  int st = best_hits(R->S, R->Den, R->n_rows, R->n_cols, 1, &R->row_ptr, &R->row_col, &R->row_best_s,
                     &R->row_best_den);
  /* A_ji: the Best Hits of every gene of G_j in G_i, i.e. of every column
   * (J is symmetric, so column k of S_ij is row k of S_ji). */
  if (st == ORC_OK)
    st = best_hits(R->S, R->Den, R->n_cols, R->n_rows, 0, &R->col_ptr, &R->col_row, &R->col_best_s,
                   &R->col_best_den);
  if (st != ORC_OK) {
    R->status = st;
    return R;
  }

  /* Algorithm 3: relevant columns, column maximum check, reciprocal check. */
  uint64_t n_row_bh = (uint64_t)R->row_ptr[R->n_rows];
  R->bbh_a = (int32_t*)malloc(sizeof(int32_t) * (n_row_bh ? n_row_bh : 1));
  R->bbh_b = (int32_t*)malloc(sizeof(int32_t) * (n_row_bh ? n_row_bh : 1));
  if (!R->bbh_a || !R->bbh_b) {
    R->status = ORC_ERR_OOM;
    return R;
  }
  R->n_bbh = 0;
  for (uint32_t k = 0; k < R->n_cols; ++k) {
    /* is column k relevant, i.e. in some A_ij[l]? and its maximum */
    uint32_t cs = R->col_best_s[k], cd = R->col_best_den[k];
    for (uint32_t l = 0; l < R->n_rows; ++l) {
      if (!contains(R->row_col, R->row_ptr[l], R->row_ptr[l + 1], (int32_t)k)) continue;
      size_t at = (size_t)l * R->n_cols + k;
      if (cs == 0 || cmp_ratio(R->S[at], R->Den[at], cs, cd) != 0) continue; /* not the column max */
      if (!contains(R->col_row, R->col_ptr[k], R->col_ptr[k + 1], (int32_t)l)) continue;
      R->bbh_a[R->n_bbh] = (int32_t)l;
      R->bbh_b[R->n_bbh] = (int32_t)k;
      R->n_bbh += 1;
    }
  }
  /* list the pairs in ascending (a, b) order: insertion sort on a (stable) */
  for (uint64_t x = 1; x < R->n_bbh; ++x) {
    int32_t a = R->bbh_a[x], b = R->bbh_b[x];
    uint64_t y = x;
    while (y > 0 && (R->bbh_a[y - 1] > a || (R->bbh_a[y - 1] == a && R->bbh_b[y - 1] > b))) {
      R->bbh_a[y] = R->bbh_a[y - 1];
      R->bbh_b[y] = R->bbh_b[y - 1];
      --y;
    }
    R->bbh_a[y] = a;
    R->bbh_b[y] = b;
  }
  R->status = ORC_OK;
  return R;
}

int orc_pair_status(const orc_pair* R) { return R->status; }

void orc_pair_sizes(const orc_pair* R, uint32_t* n_rows, uint32_t* n_cols, uint64_t* n_row_bh,
                    uint64_t* n_col_bh, uint64_t* n_bbh) {
  *n_rows = R->n_rows;
  *n_cols = R->n_cols;
  *n_row_bh = R->row_ptr ? (uint64_t)R->row_ptr[R->n_rows] : 0;
  *n_col_bh = R->col_ptr ? (uint64_t)R->col_ptr[R->n_cols] : 0;
  *n_bbh = R->n_bbh;
}

void orc_pair_matrix(const orc_pair* R, uint32_t* S, uint32_t* Den) {
  size_t cells = (size_t)R->n_rows * R->n_cols;
  if (S) memcpy(S, R->S, sizeof(uint32_t) * cells);
  if (Den) memcpy(Den, R->Den, sizeof(uint32_t) * cells);
}

void orc_pair_row_bh(const orc_pair* R, int64_t* ptr, int32_t* col, uint32_t* best_s, uint32_t* best_den) {
  memcpy(ptr, R->row_ptr, sizeof(int64_t) * ((size_t)R->n_rows + 1));
  memcpy(col, R->row_col, sizeof(int32_t) * (size_t)R->row_ptr[R->n_rows]);
  memcpy(best_s, R->row_best_s, sizeof(uint32_t) * R->n_rows);
  memcpy(best_den, R->row_best_den, sizeof(uint32_t) * R->n_rows);
}

void orc_pair_col_bh(const orc_pair* R, int64_t* ptr, int32_t* row, uint32_t* best_s, uint32_t* best_den) {
  memcpy(ptr, R->col_ptr, sizeof(int64_t) * ((size_t)R->n_cols + 1));
  memcpy(row, R->col_row, sizeof(int32_t) * (size_t)R->col_ptr[R->n_cols]);
  memcpy(best_s, R->col_best_s, sizeof(uint32_t) * R->n_cols);
  memcpy(best_den, R->col_best_den, sizeof(uint32_t) * R->n_cols);
}

void orc_pair_bbh(const orc_pair* R, int32_t* a, int32_t* b) {
  memcpy(a, R->bbh_a, sizeof(int32_t) * R->n_bbh);
  memcpy(b, R->bbh_b, sizeof(int32_t) * R->n_bbh);
}
