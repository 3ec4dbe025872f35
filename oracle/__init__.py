"""CPU oracle of the PanDelos-plus hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import this package.  The product (the CUDA library and its binding) never
does; the two share no code.

The arithmetic lives in ``pd_oracle.c`` (plain C, compiled here with gcc);
this module builds it and marshals numpy arrays through ctypes.  Every
function follows the passage of the paper named in its docstring:

* ``choose_k``     Eq. (4), read as the smallest k with 20^k >= total residues
                   (PARITY UNPINNED: the paper prints no k for any dataset);
* ``Profiles``     Eqs. (1)-(3) and Algorithm 1 (multiplicity vectors);
* ``summin``       Eq. (5) numerator and denominator of one gene pair;
* ``pair``         Algorithm 2 (S_ij, Best Hits of rows, Eq. (8)) and
                   Algorithm 3 (Bidirectional Best Hits, Eq. (9));
* ``families``     phase (c): connected components of the BBH graph;
* ``paralog_hits`` Eq. (8) within one genome (the gene itself excluded);
* ``filtered_pair`` Algorithms 2-3 with the theta and tau filters of Eqs. (6)-(7).

A second, independent oracle (``pd_oracle_b.c``, no code shared with
``pd_oracle.c``) walks an inverted index with a pool of host threads over the
query genes -- the paper's own data decomposition ("Parallel implementation")
-- and reaches the same integers fast enough to check whole datasets:

* ``IndexB``       Eq. (1) and Algorithm 1 (codes, multiplicity vectors) plus
                   the inverted index of the dataset;
* ``best_hits_b``  Eq. (5) numerators by posting walk, Eq. (8) Best Hits of
                   listed query genes towards listed genomes;
* ``all_pairs_b``  every gene's Best Hits in every other genome and the BBH
                   pairs of every genome pair (Eq. (9), Algorithm 3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libpd_oracle.so")
_SRC_B = os.path.join(_HERE, "pd_oracle_b.c")
_LIB_B = os.path.join(_HERE, "_build", "libpd_oracle_b.so")
# A test may point the loader at another compiled copy (used to check that the
# pins reject deliberately broken oracles).
_LIB_OVERRIDE = os.environ.get("PD_ORACLE_LIB")
_lock = threading.Lock()
_lib = None
_lib_b = None

OK, ERR_ARG, ERR_ALPHABET, ERR_IDENTITY, ERR_OOM = 0, 1, 2, 3, 4


def _compile(src: str, lib: str, force: bool) -> str:
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread", "-o", tmp, src])
        os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Compile pd_oracle.c and pd_oracle_b.c into two shared libraries (gcc, plain C11)."""
    _compile(_SRC_B, _LIB_B, force)
    return _compile(_SRC, _LIB, force)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(_LIB_OVERRIDE if _LIB_OVERRIDE else build())
        P, u8p, i64p, i32p, u32p = C.c_void_p, C.POINTER(C.c_uint8), C.POINTER(C.c_int64), \
            C.POINTER(C.c_int32), C.POINTER(C.c_uint32)
        lib.orc_choose_k.restype = C.c_int
        lib.orc_choose_k.argtypes = [C.c_uint64, C.c_int]
        lib.orc_build.restype = P
        lib.orc_build.argtypes = [u8p, C.c_uint64, i64p, C.c_uint32, C.c_int, C.POINTER(C.c_int)]
        lib.orc_directional.restype = C.c_int
        lib.orc_directional.argtypes = [P, C.c_uint32, C.c_uint32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        lib.orc_build_alphabet.restype = P
        lib.orc_build_alphabet.argtypes = [u8p, C.c_uint64, i64p, C.c_uint32, C.c_int, C.c_int, C.POINTER(C.c_int)]
        lib.orc_free.argtypes = [P]
        lib.orc_mv_len.restype = C.c_uint32
        lib.orc_mv_len.argtypes = [P, C.c_uint32]
        lib.orc_La.restype = C.c_uint32
        lib.orc_La.argtypes = [P, C.c_uint32]
        lib.orc_mv_get.argtypes = [P, C.c_uint32, u8p, u32p]
        lib.orc_summin.restype = C.c_int
        lib.orc_summin.argtypes = [P, C.c_uint32, C.c_uint32, u32p, u32p]
        lib.orc_pair_run.restype = P
        lib.orc_pair_run.argtypes = [P, i32p, C.c_uint32, C.c_uint32, C.c_int]
        lib.orc_pair_status.restype = C.c_int
        lib.orc_pair_status.argtypes = [P]
        lib.orc_pair_free.argtypes = [P]
        lib.orc_pair_sizes.argtypes = [P, u32p, u32p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                       C.POINTER(C.c_uint64)]
        lib.orc_pair_matrix.argtypes = [P, u32p, u32p]
        lib.orc_pair_row_bh.argtypes = [P, i64p, i32p, u32p, u32p]
        lib.orc_pair_col_bh.argtypes = [P, i64p, i32p, u32p, u32p]
        lib.orc_pair_bbh.argtypes = [P, i32p, i32p]
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def choose_k(total_residues: int, alphabet: int = 20) -> int:
    """Eq. (4) reading: smallest k with alphabet**k >= total residues."""
    return int(_load().orc_choose_k(int(total_residues), int(alphabet)))


class Profiles:
    """Multiplicity vectors of every gene of a dataset (Algorithm 1)."""

    def __init__(self, residues: np.ndarray, gene_ptr: np.ndarray, k: int, alphabet: int = 20):
        lib = _load()
        self._res = np.ascontiguousarray(residues, dtype=np.uint8)
        self._gptr = np.ascontiguousarray(gene_ptr, dtype=np.int64)
        self.k = int(k)
        self.n_genes = int(self._gptr.shape[0] - 1)
        st = C.c_int(0)
        res = self._res if self._res.size else np.zeros(1, np.uint8)
        self._h = lib.orc_build_alphabet(_ptr(res, C.c_uint8), self._res.size, _ptr(self._gptr, C.c_int64),
                                         self.n_genes, self.k, int(alphabet), C.byref(st))
        if not self._h:
            raise OracleError(st.value, "build")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_free(h)
            self._h = None

    def La(self, g: int) -> int:
        """Number of windows of gene g: |g|-k+1, or 0 when |g| < k."""
        return int(_lib.orc_La(self._h, g))

    def mv(self, g: int):
        """(k-mer strings as bytes, counts) of gene g, ascending by k-mer."""
        n = int(_lib.orc_mv_len(self._h, g))
        kmers = np.zeros(max(1, n * self.k), np.uint8)
        cnt = np.zeros(max(1, n), np.uint32)
        _lib.orc_mv_get(self._h, g, _ptr(kmers, C.c_uint8), _ptr(cnt, C.c_uint32))
        kb = kmers[: n * self.k].tobytes()
        return [kb[e * self.k:(e + 1) * self.k] for e in range(n)], cnt[:n].copy()

    def directional(self, a: int, b: int):
        """Eq. (7) numerators: (sum of mult_a, sum of mult_b) over the shared k-mers."""
        x, y = C.c_uint32(0), C.c_uint32(0)
        st = _lib.orc_directional(self._h, a, b, C.byref(x), C.byref(y))
        if st != OK:
            raise OracleError(st, "directional")
        return x.value, y.value

    def summin(self, a: int, b: int):
        """(sum of min(mult) over shared k-mers, sum of max(mult) over the union)."""
        s, d = C.c_uint32(0), C.c_uint32(0)
        st = _lib.orc_summin(self._h, a, b, C.byref(s), C.byref(d))
        if st != OK:
            raise OracleError(st, "summin")
        return int(s.value), int(d.value)


@dataclass
class PairResult:
    """One genome pair (G_i rows, G_j columns); gene indices are local."""
    S: np.ndarray          # uint32 [n_rows, n_cols]: sum min (Eq. (5) numerator)
    Den: np.ndarray        # uint32 [n_rows, n_cols]: sum max (Eq. (5) denominator)
    row_ptr: np.ndarray    # int64 [n_rows+1]: A_ij as CSR
    row_col: np.ndarray    # int32
    row_best_s: np.ndarray
    row_best_den: np.ndarray
    col_ptr: np.ndarray    # int64 [n_cols+1]: A_ji as CSR
    col_row: np.ndarray
    col_best_s: np.ndarray
    col_best_den: np.ndarray
    bbh: np.ndarray        # int32 [n_bbh, 2]: (a, b) ascending

    def row_bh(self, a: int):
        return self.row_col[self.row_ptr[a]:self.row_ptr[a + 1]]

    def col_bh(self, b: int):
        return self.col_row[self.col_ptr[b]:self.col_ptr[b + 1]]


def pair(prof: Profiles, genome_ptr: np.ndarray, gi: int, gj: int, n_threads: int = 1) -> PairResult:
    """Algorithms 2 and 3 for genomes gi (rows) and gj (columns)."""
    lib = _load()
    gp = np.ascontiguousarray(genome_ptr, dtype=np.int32)
    h = lib.orc_pair_run(prof._h, _ptr(gp, C.c_int32), gi, gj, int(n_threads))
    if not h:
        raise OracleError(ERR_OOM, "pair")
    try:
        st = lib.orc_pair_status(h)
        if st != OK:
            raise OracleError(st, "pair")
        nr, nc = C.c_uint32(0), C.c_uint32(0)
        nrb, ncb, nbbh = C.c_uint64(0), C.c_uint64(0), C.c_uint64(0)
        lib.orc_pair_sizes(h, C.byref(nr), C.byref(nc), C.byref(nrb), C.byref(ncb), C.byref(nbbh))
        nr, nc, nrb, ncb, nbbh = nr.value, nc.value, nrb.value, ncb.value, nbbh.value
        S = np.zeros((max(nr, 1), max(nc, 1)), np.uint32)
        D = np.zeros_like(S)
        lib.orc_pair_matrix(h, _ptr(S, C.c_uint32), _ptr(D, C.c_uint32))
        rp = np.zeros(nr + 1, np.int64)
        rc = np.zeros(max(nrb, 1), np.int32)
        rbs = np.zeros(max(nr, 1), np.uint32)
        rbd = np.zeros(max(nr, 1), np.uint32)
        lib.orc_pair_row_bh(h, _ptr(rp, C.c_int64), _ptr(rc, C.c_int32), _ptr(rbs, C.c_uint32),
                            _ptr(rbd, C.c_uint32))
        cp = np.zeros(nc + 1, np.int64)
        cr = np.zeros(max(ncb, 1), np.int32)
        cbs = np.zeros(max(nc, 1), np.uint32)
        cbd = np.zeros(max(nc, 1), np.uint32)
        lib.orc_pair_col_bh(h, _ptr(cp, C.c_int64), _ptr(cr, C.c_int32), _ptr(cbs, C.c_uint32),
                            _ptr(cbd, C.c_uint32))
        ba = np.zeros(max(nbbh, 1), np.int32)
        bb = np.zeros(max(nbbh, 1), np.int32)
        lib.orc_pair_bbh(h, _ptr(ba, C.c_int32), _ptr(bb, C.c_int32))
        return PairResult(S=S[:nr, :nc], Den=D[:nr, :nc], row_ptr=rp, row_col=rc[:nrb],
                          row_best_s=rbs[:nr], row_best_den=rbd[:nr], col_ptr=cp, col_row=cr[:ncb],
                          col_best_s=cbs[:nc], col_best_den=cbd[:nc],
                          bbh=np.stack([ba[:nbbh], bb[:nbbh]], axis=1))
    finally:
        lib.orc_pair_free(h)


def pair_for_dataset(ds, gi: int, gj: int, k: int, n_threads: int = 1, alphabet: int = 20) -> PairResult:
    """Algorithms 1-3 on genomes gi and gj of a dataset (only their genes are profiled)."""
    sub = ds.subset([gi, gj]) if gi != gj else ds.subset([gi])
    prof = Profiles(sub.residues, sub.gene_ptr, k, alphabet)
    if gi == gj:
        return pair(prof, sub.genome_ptr, 0, 0, n_threads)
    return pair(prof, sub.genome_ptr, 0, 1, n_threads)


def all_pairs_bbh(ds, k: int, n_threads: int = 1) -> np.ndarray:
    """Algorithm 3 on every genome pair i < j of a dataset: BBH pairs (a, b)
    as global gene ids, genome(a) < genome(b), ascending."""
    gp = ds.genome_ptr
    out = []
    for i in range(ds.n_genomes):
        for j in range(i + 1, ds.n_genomes):
            R = pair_for_dataset(ds, i, j, k, n_threads)
            if len(R.bbh):
                out.append(R.bbh.astype(np.int64) + [int(gp[i]), int(gp[j])])
    if not out:
        return np.zeros((0, 2), np.int64)
    pairs = np.concatenate(out)
    return pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]


def families(n_nodes: int, pairs) -> np.ndarray:
    """Phase (c), "extract gene families from the Bidirectional Best Hits",
    read as the connected components of the BBH graph (the refinement
    PanDelos applies afterwards is not specified).  Breadth-first search from
    every unvisited node in ascending order, so the first node of each
    component -- its label -- is the component's smallest id."""
    adj = [[] for _ in range(n_nodes)]
    for a, b in pairs:
        adj[int(a)].append(int(b))
        adj[int(b)].append(int(a))
    label = np.full(n_nodes, -1, np.int64)
    for s in range(n_nodes):
        if label[s] >= 0:
            continue
        label[s] = s
        frontier = [s]
        while frontier:
            nxt = []
            for u in frontier:
                for v in adj[u]:
                    if label[v] < 0:
                        label[v] = s
                        nxt.append(v)
            frontier = nxt
    return label


def paralog_hits(ds, k: int, n_threads: int = 1):
    """Eq. (8) inside each genome with the gene itself excluded (the
    within-genome comparison): for every gene a of genome G_i, the genes b of
    G_i, b != a, with s(a, b) >= 1 that maximise s / sum-max, ties kept.
    Uses the oracle's own S and sum-max matrices of the pair (G_i, G_i).
    Returns one (columns, s values) per gene, columns as global gene ids."""
    gp = ds.genome_ptr
    rows = []
    for i in range(ds.n_genomes):
        g0 = int(gp[i])
        n = int(gp[i + 1] - gp[i])
        R = pair_for_dataset(ds, i, i, k, n_threads) if n else None
        for a in range(n):
            best, hits = None, []
            for b in range(n):
                s = int(R.S[a, b])
                if b == a or s < 1:
                    continue
                den = int(R.Den[a, b])
                if best is None or s * best[1] > best[0] * den:
                    best, hits = (s, den), [b]
                elif s * best[1] == best[0] * den:
                    hits.append(b)
            rows.append(([g0 + b for b in hits], [int(R.S[a, b]) for b in hits]))
    return rows


def paralog_bbh(rows):
    """Eq. (9) inside a genome: pairs (a, b), a < b, each a Best Hit of the other."""
    sets = [set(c) for c, _ in rows]
    return [(a, b) for a in range(len(rows)) for b in sorted(sets[a]) if b > a and a in sets[b]]


def filtered_pair(ds, gi: int, gj: int, k: int, theta=(0, 1), tau=(0, 1), alphabet: int = 20):
    """Algorithms 2-3 for genomes gi, gj with the candidate filters of Eq. (6)
    (length ratio theta) and Eq. (7) (directional similarity tau) applied
    before the Best Hit argmax; theta and tau are (numerator, denominator),
    numerator 0 = off.  Returns (row Best Hits, column Best Hits, BBH pairs) as
    lists of local indices."""
    sub = ds.subset([gi, gj])
    prof = Profiles(sub.residues, sub.gene_ptr, k, alphabet)
    R = pair(prof, sub.genome_ptr, 0, 1)
    n_a, n_b = R.S.shape
    glen = np.diff(sub.gene_ptr).astype(np.int64)

    def candidate(a, b):
        s = int(R.S[a, b])
        if s < 1:
            return False
        la, lb = int(glen[a]), int(glen[n_a + b])
        if theta[0] and (la * theta[1] < theta[0] * lb or lb * theta[1] < theta[0] * la):
            return False
        if tau[0]:
            pa, pb = prof.directional(a, n_a + b)
            if pa * tau[1] < tau[0] * (la - k + 1) or pb * tau[1] < tau[0] * (lb - k + 1):
                return False
        return True

    cand = [[candidate(a, b) for b in range(n_b)] for a in range(n_a)]

    def best_set(pairs):  # [(index, s, den)] -> indices at the maximum s / den
        best, out = None, []
        for x, s, d in pairs:
            if best is None or s * best[1] > best[0] * d:
                best, out = (s, d), [x]
            elif s * best[1] == best[0] * d:
                out.append(x)
        return out

    rows = [best_set([(b, int(R.S[a, b]), int(R.Den[a, b])) for b in range(n_b) if cand[a][b]]) for a in range(n_a)]
    cols = [best_set([(a, int(R.S[a, b]), int(R.Den[a, b])) for a in range(n_a) if cand[a][b]]) for b in range(n_b)]
    bbh = [(a, b) for a in range(n_a) for b in rows[a] if a in cols[b]]
    return rows, cols, bbh


# --------------------------------------------------------------------------- oracle B
def _load_b():
    global _lib_b
    with _lock:
        if _lib_b is not None:
            return _lib_b
        override = os.environ.get("PD_ORACLE_B_LIB")  # a test may load a deliberately broken copy
        lib = C.CDLL(override if override else _compile(_SRC_B, _LIB_B, False))
        P, u8p, i64p, i32p, u32p = C.c_void_p, C.POINTER(C.c_uint8), C.POINTER(C.c_int64), \
            C.POINTER(C.c_int32), C.POINTER(C.c_uint32)
        lib.orb_build.restype = P
        lib.orb_build.argtypes = [u8p, C.c_uint64, i64p, C.c_uint32, i32p, C.c_uint32, C.c_int, C.c_int, C.c_int,
                                  C.POINTER(C.c_int)]
        lib.orb_free.argtypes = [P]
        lib.orb_n_entries.restype = C.c_uint64
        lib.orb_n_entries.argtypes = [P]
        lib.orb_n_lists.restype = C.c_uint64
        lib.orb_n_lists.argtypes = [P]
        lib.orb_La.restype = C.c_uint32
        lib.orb_La.argtypes = [P, C.c_uint32]
        lib.orb_best_hits.restype = P
        lib.orb_best_hits.argtypes = [P, u32p, C.c_uint32, u8p, C.c_int, C.c_int, C.POINTER(C.c_int)]
        lib.orb_hits_free.argtypes = [P]
        lib.orb_hits_rows.restype = C.c_uint32
        lib.orb_hits_rows.argtypes = [P]
        lib.orb_hits_count.restype = C.c_uint64
        lib.orb_hits_count.argtypes = [P]
        lib.orb_hits_get.argtypes = [P, i64p, i32p, u32p]
        lib.orb_bbh.restype = C.c_uint64
        lib.orb_bbh.argtypes = [P, P, i32p, i32p, C.c_uint64]
        _lib_b = lib
        return lib


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 4


class IndexB:
    """Oracle B over a whole dataset: multiplicity vectors (Algorithm 1) and
    the inverted index (for every k-mer, its genes ascending)."""

    def __init__(self, ds, k: int, alphabet: int = 20, n_threads: int = 0):
        lib = _load_b()
        self._res = np.ascontiguousarray(ds.residues, dtype=np.uint8)
        self._gptr = np.ascontiguousarray(ds.gene_ptr, dtype=np.int64)
        self.genome_ptr = np.ascontiguousarray(ds.genome_ptr, dtype=np.int32)
        self.k, self.alphabet = int(k), int(alphabet)
        self.n_genes = int(self._gptr.shape[0] - 1)
        self.n_genomes = int(self.genome_ptr.shape[0] - 1)
        self.n_threads = int(n_threads) or default_threads()
        st = C.c_int(0)
        res = self._res if self._res.size else np.zeros(1, np.uint8)
        self._h = lib.orb_build(_ptr(res, C.c_uint8), self._res.size, _ptr(self._gptr, C.c_int64), self.n_genes,
                                _ptr(self.genome_ptr, C.c_int32), self.n_genomes, self.k, self.alphabet,
                                self.n_threads, C.byref(st))
        if not self._h:
            raise OracleError(st.value, "oracle B build")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib_b is not None:
            _lib_b.orb_free(h)
            self._h = None

    @property
    def n_entries(self) -> int:
        return int(_lib_b.orb_n_entries(self._h))

    def La(self, g: int) -> int:
        return int(_lib_b.orb_La(self._h, g))


def _hits_b(idx: IndexB, queries, targets=None, own_genome: bool = False):
    lib = _load_b()
    q = np.ascontiguousarray(queries, dtype=np.uint32)
    qq = q if q.size else np.zeros(1, np.uint32)
    mask = None
    if targets is not None:
        m = np.zeros(idx.n_genomes, np.uint8)
        m[np.asarray(list(targets), dtype=np.int64)] = 1
        mask = _ptr(m, C.c_uint8)
    st = C.c_int(0)
    h = lib.orb_best_hits(idx._h, _ptr(qq, C.c_uint32), q.size, mask, 1 if own_genome else 0, idx.n_threads,
                          C.byref(st))
    if not h:
        raise OracleError(st.value, "oracle B best hits")
    return h


def best_hits_b(idx: IndexB, queries, targets=None, own_genome: bool = False):
    """Eq. (8) Best Hits of the listed query genes (global ids) in each target
    genome (``targets``: genome indices; None = every genome but the query's
    own; ``own_genome`` adds the query's genome, the gene itself excluded).
    Returns (row_ptr int64[n_q+1], cols int32 global gene ids ascending per
    row, s uint32 sum-min)."""
    lib = _load_b()
    h = _hits_b(idx, queries, targets, own_genome)
    try:
        n = int(lib.orb_hits_count(h))
        nr = int(lib.orb_hits_rows(h))
        rp = np.zeros(nr + 1, np.int64)
        cols = np.zeros(max(n, 1), np.int32)
        s = np.zeros(max(n, 1), np.uint32)
        lib.orb_hits_get(h, _ptr(rp, C.c_int64), _ptr(cols, C.c_int32), _ptr(s, C.c_uint32))
        return rp, cols[:n], s[:n]
    finally:
        lib.orb_hits_free(h)


def all_pairs_b(idx: IndexB):
    """Algorithms 2-3 over every genome pair: (row_ptr, cols, s) of every
    gene's Best Hits in every other genome (rows in gene order) and the BBH
    pairs (a, b) with genome(a) < genome(b), ascending (int32 [n, 2])."""
    lib = _load_b()
    h = _hits_b(idx, np.arange(idx.n_genes, dtype=np.uint32))
    try:
        n = int(lib.orb_hits_count(h))
        rp = np.zeros(idx.n_genes + 1, np.int64)
        cols = np.zeros(max(n, 1), np.int32)
        s = np.zeros(max(n, 1), np.uint32)
        lib.orb_hits_get(h, _ptr(rp, C.c_int64), _ptr(cols, C.c_int32), _ptr(s, C.c_uint32))
        nb = int(lib.orb_bbh(idx._h, h, None, None, 0))
        a = np.zeros(max(nb, 1), np.int32)
        b = np.zeros(max(nb, 1), np.int32)
        lib.orb_bbh(idx._h, h, _ptr(a, C.c_int32), _ptr(b, C.c_int32), nb)
        return rp, cols[:n], s[:n], np.stack([a[:nb], b[:nb]], axis=1)
    finally:
        lib.orb_hits_free(h)
