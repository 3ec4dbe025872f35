"""Seeded synthetic pangenomes (amino-acid genomes made of mutated gene families).

This module only *generates input*: it draws residues, gene boundaries and
genome boundaries.  It contains none of the similarity method's arithmetic
(no k-mers, no multiplicities, no Jaccard), so that both the CPU oracle and the
CUDA path can read the same seeded inputs without sharing any method code.

Model (a stand-in for the paper's PANPROVA collections, "Dataset construction"
and Table 2, whose genomes are not available here):

* a fixed amino-acid background composition (20 letters, ``ALPHABET`` order);
* ``n_families`` ancestral family sequences drawn i.i.d. from the background;
  each family has a substitution rate ``U[0, subst_max]`` and an indel rate
  ``U[0, indel_max]``;
* each genome holds copies of core families (present in every genome), a
  random draw of accessory families, paralog copies (extra copies of families
  the genome already holds) and singleton genes (fresh random sequences);
* each copy evolves independently from its family's ancestor: every residue is
  substituted with the family's substitution rate (new letter drawn from the
  background) and every position carries a single-residue deletion with
  probability ``indel/2`` and a single-residue insertion after it with
  probability ``indel/2``;
* gene order inside a genome is a random permutation.

Everything is driven by one ``numpy.random.Generator(PCG64(seed))`` stream.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ALPHABET = b"ACDEFGHIKLMNPQRSTVWY"

# Approximate amino-acid composition of curated protein databases (percent).
_BACKGROUND_PCT = {
    "A": 8.25, "R": 5.53, "N": 4.06, "D": 5.45, "C": 1.37, "Q": 3.93,
    "E": 6.75, "G": 7.07, "H": 2.27, "I": 5.96, "L": 9.66, "K": 5.84,
    "M": 2.42, "F": 3.86, "P": 4.70, "S": 6.56, "T": 5.34, "W": 1.08,
    "Y": 2.92, "V": 6.87,
}
BACKGROUND = np.array([_BACKGROUND_PCT[chr(c)] for c in ALPHABET], dtype=np.float64)
BACKGROUND /= BACKGROUND.sum()
_LETTERS = np.frombuffer(ALPHABET, dtype=np.uint8)

# Nucleotide datasets: ACGT with 50% GC content.
NT_ALPHABET = b"ACGT"
NT_BACKGROUND = np.array([0.25, 0.25, 0.25, 0.25])
_NT_LETTERS = np.frombuffer(NT_ALPHABET, dtype=np.uint8)


@dataclass
class Pangenome:
    """A dataset of genomes; genes are ASCII amino-acid strings.

    residues   uint8[N]    all genes concatenated (ASCII letters)
    gene_ptr   int64[G+1]  gene g is residues[gene_ptr[g]:gene_ptr[g+1]]
    genome_ptr int32[n+1]  genome i holds genes genome_ptr[i] .. genome_ptr[i+1]-1
    family     int32[G]    generating family per gene (-1 for singletons); a
                           sanity label only, never an input of the method
    """

    residues: np.ndarray
    gene_ptr: np.ndarray
    genome_ptr: np.ndarray
    family: np.ndarray
    name: str = ""
    params: dict = field(default_factory=dict)

    @property
    def n_genes(self) -> int:
        return int(self.gene_ptr.shape[0] - 1)

    @property
    def n_genomes(self) -> int:
        return int(self.genome_ptr.shape[0] - 1)

    @property
    def n_residues(self) -> int:
        return int(self.residues.shape[0])

    def genome_sizes(self) -> np.ndarray:
        return np.diff(self.genome_ptr).astype(np.int64)

    def gene(self, g: int) -> bytes:
        return self.residues[self.gene_ptr[g]:self.gene_ptr[g + 1]].tobytes()

    def logical_pairs(self) -> int:
        """Number of cross-genome gene pairs sum_{i<j} |G_i| |G_j|."""
        s = self.genome_sizes()
        return int((s.sum() ** 2 - (s * s).sum()) // 2)

    def subset(self, genomes) -> "Pangenome":
        """The dataset restricted to the listed genomes (in the given order)."""
        parts, gptr, fam, gnm = [], [0], [], [0]
        for i in genomes:
            g0, g1 = int(self.genome_ptr[i]), int(self.genome_ptr[i + 1])
            r0, r1 = int(self.gene_ptr[g0]), int(self.gene_ptr[g1])
            parts.append(self.residues[r0:r1])
            base = gptr[-1]
            gptr.extend((self.gene_ptr[g0 + 1:g1 + 1] - r0 + base).tolist())
            fam.append(self.family[g0:g1])
            gnm.append(gnm[-1] + (g1 - g0))
        return Pangenome(
            residues=np.concatenate(parts) if parts else np.zeros(0, np.uint8),
            gene_ptr=np.asarray(gptr, dtype=np.int64),
            genome_ptr=np.asarray(gnm, dtype=np.int32),
            family=np.concatenate(fam) if fam else np.zeros(0, np.int32),
            name=f"{self.name}[{','.join(map(str, genomes))}]",
            params=self.params,
        )


def from_strings(genomes) -> Pangenome:
    """Build a dataset from explicit gene strings: ``[[b"ACD..", ...], ...]``."""
    res, gptr, gnm = [], [0], [0]
    for genes in genomes:
        for s in genes:
            b = s.encode() if isinstance(s, str) else bytes(s)
            res.append(b)
            gptr.append(gptr[-1] + len(b))
        gnm.append(gnm[-1] + len(genes))
    raw = b"".join(res)
    return Pangenome(
        residues=np.frombuffer(raw, dtype=np.uint8).copy() if raw else np.zeros(0, np.uint8),
        gene_ptr=np.asarray(gptr, dtype=np.int64),
        genome_ptr=np.asarray(gnm, dtype=np.int32),
        family=np.full(gptr.__len__() - 1, -1, dtype=np.int32),
        name="strings",
    )


# ---------------------------------------------------------------------------
# length distributions
# ---------------------------------------------------------------------------

def _lengths(rng, n, dist):
    kind = dist[0]
    if kind == "uniform":
        lo, hi = dist[1], dist[2]
        return rng.integers(lo, hi + 1, size=n, dtype=np.int64)
    if kind == "lognormal":
        median, sigma, lo, hi = dist[1], dist[2], dist[3], dist[4]
        x = rng.lognormal(mean=np.log(median), sigma=sigma, size=n)
        return np.clip(np.rint(x), lo, hi).astype(np.int64)
    raise ValueError(f"unknown length distribution {dist!r}")


def _random_codes(rng, n, bg=BACKGROUND):
    return rng.choice(len(bg), size=n, p=bg).astype(np.uint8)


def generate(
    *,
    n_genomes: int,
    genes_per_genome,
    n_families: int,
    length_dist,
    core_frac: float,
    accessory_draw: float | None,
    subst_max: float,
    indel_max: float,
    paralog_frac: float,
    singleton_frac: float,
    seed: int,
    name: str = "",
    alphabet: str = "aa",
) -> Pangenome:
    """Draw a seeded pangenome.

    genes_per_genome  ("fixed", m), ("poisson", mean) or ("list", [m_0, m_1, ...])
    accessory_draw    if set, the fraction of *all* families each genome draws
                      (no core set; used by the 4-genome workload); otherwise
                      every genome holds all core families and fills up to its
                      gene count with accessory families drawn without
                      replacement from the non-core ones.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    bg, letters = (BACKGROUND, _LETTERS) if alphabet == "aa" else (NT_BACKGROUND, _NT_LETTERS)
    fam_len = _lengths(rng, n_families, length_dist)
    fam_ptr = np.zeros(n_families + 1, dtype=np.int64)
    np.cumsum(fam_len, out=fam_ptr[1:])
    fam_seq = _random_codes(rng, int(fam_ptr[-1]), bg)
    fam_sub = rng.uniform(0.0, subst_max, size=n_families)
    fam_indel = rng.uniform(0.0, indel_max, size=n_families)
    n_core = int(round(core_frac * n_families))
    core = np.arange(n_core)
    accessory_pool = np.arange(n_core, n_families)

    # ---- gene specs: (family or -1) per gene, genome by genome
    specs = []
    gnm = [0]
    for _ in range(n_genomes):
        if genes_per_genome[0] == "fixed":
            m = int(genes_per_genome[1])
        elif genes_per_genome[0] == "list":
            m = int(genes_per_genome[1][len(specs)])
        else:
            m = int(rng.poisson(genes_per_genome[1]))
        n_single = int(round(singleton_frac * m))
        if accessory_draw is not None:
            drawn = rng.choice(n_families, size=int(round(accessory_draw * n_families)), replace=False)
        else:
            n_para0 = int(round(paralog_frac * m))
            n_acc = max(0, min(len(accessory_pool), m - n_single - n_para0 - n_core))
            drawn = np.concatenate([core, rng.choice(accessory_pool, size=n_acc, replace=False)])
        n_fill = max(0, m - n_single - len(drawn))
        para = rng.choice(drawn, size=n_fill, replace=True) if len(drawn) else np.zeros(0, np.int64)
        fams = np.concatenate([drawn, para, np.full(n_single, -1)]).astype(np.int64)
        fams = fams[rng.permutation(len(fams))]
        specs.append(fams)
        gnm.append(gnm[-1] + len(fams))
    family = np.concatenate(specs) if specs else np.zeros(0, np.int64)
    G = len(family)

    # ---- source sequences (ancestral copy or fresh singleton)
    is_single = family < 0
    src_len = np.where(is_single, 0, fam_len[np.maximum(family, 0)])
    single_len = _lengths(rng, int(is_single.sum()), length_dist)
    src_len[is_single] = single_len
    src_ptr = np.zeros(G + 1, dtype=np.int64)
    np.cumsum(src_len, out=src_ptr[1:])
    N0 = int(src_ptr[-1])
    # index of every source residue in fam_seq (or -1 for singleton residues)
    gene_of = np.repeat(np.arange(G), src_len)
    pos_in_gene = np.arange(N0, dtype=np.int64) - src_ptr[gene_of]
    fam_of = family[gene_of]
    src = np.empty(N0, dtype=np.uint8)
    fam_mask = fam_of >= 0
    src[fam_mask] = fam_seq[fam_ptr[fam_of[fam_mask]] + pos_in_gene[fam_mask]]
    src[~fam_mask] = _random_codes(rng, int((~fam_mask).sum()), bg)

    # ---- substitutions (family copies only)
    sub_rate = np.where(fam_mask, fam_sub[np.maximum(fam_of, 0)], 0.0)
    hit = rng.random(N0) < sub_rate
    src[hit] = _random_codes(rng, int(hit.sum()), bg)

    # ---- single-residue indels (family copies only)
    indel_rate = np.where(fam_mask, fam_indel[np.maximum(fam_of, 0)], 0.0)
    u = rng.random(N0)
    delete = u < indel_rate * 0.5
    insert = (u >= indel_rate * 0.5) & (u < indel_rate)
    reps = 1 - delete.astype(np.int64) + insert.astype(np.int64)
    out = np.repeat(src, reps)
    # the second copy of an inserted position becomes a fresh random residue
    first = np.zeros(N0 + 1, dtype=np.int64)
    np.cumsum(reps, out=first[1:])
    ins_slots = first[:-1][insert] + 1
    out[ins_slots] = _random_codes(rng, len(ins_slots), bg)
    new_len = np.add.reduceat(reps, src_ptr[:-1]) if G else np.zeros(0, np.int64)
    new_len = np.where(src_len > 0, new_len, 0)

    gene_ptr = np.zeros(G + 1, dtype=np.int64)
    np.cumsum(new_len, out=gene_ptr[1:])
    return Pangenome(
        residues=letters[out],
        gene_ptr=gene_ptr,
        genome_ptr=np.asarray(gnm, dtype=np.int32),
        family=family.astype(np.int32),
        name=name,
        params=dict(n_genomes=n_genomes, genes_per_genome=genes_per_genome, n_families=n_families,
                    length_dist=length_dist, core_frac=core_frac, accessory_draw=accessory_draw,
                    subst_max=subst_max, indel_max=indel_max, paralog_frac=paralog_frac,
                    singleton_frac=singleton_frac, seed=seed, alphabet=alphabet),
    )


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

WORKLOADS = {
    # 4 genomes x 250 genes, 200 families with lengths U[80,600]; each genome
    # draws 80% of the families, substitution U[0,15%], indels U[0,3%],
    # 5% singletons; the remaining genes are paralog copies.
    "pan4x250": dict(n_genomes=4, genes_per_genome=("fixed", 250), n_families=200,
                     length_dist=("uniform", 80, 600), core_frac=0.0, accessory_draw=0.8,
                     subst_max=0.15, indel_max=0.03, paralog_frac=0.0, singleton_frac=0.05,
                     seed=1),
    # 50 genomes x Poisson(3000) genes, log-normal lengths (median 300 aa,
    # sigma 0.5, clipped to 30..2500), 4000 families with 40% core,
    # substitution U[0,30%], indels U[0,5%], 10% paralogs, 5% singletons.
    "pan50x3000": dict(n_genomes=50, genes_per_genome=("poisson", 3000), n_families=4000,
                       length_dist=("lognormal", 300, 0.5, 30, 2500), core_frac=0.4,
                       accessory_draw=None, subst_max=0.30, indel_max=0.05, paralog_frac=0.10,
                       singleton_frac=0.05, seed=2),
    # 200 genomes x Poisson(4000) genes, same model with 12000 families, 25% core.
    "pan200x4000": dict(n_genomes=200, genes_per_genome=("poisson", 4000), n_families=12000,
                        length_dist=("lognormal", 300, 0.5, 30, 2500), core_frac=0.25,
                        accessory_draw=None, subst_max=0.30, indel_max=0.05, paralog_frac=0.10,
                        singleton_frac=0.05, seed=3),
    # The pan200x4000 model at a quarter of the genes (Poisson(1000) genes per
    # genome, 3000 families): the same 200 genomes and k = 7, so posting lists
    # of the same lengths and the same walk, in a case small enough for
    # counter captures.
    "pan200x1000": dict(n_genomes=200, genes_per_genome=("poisson", 1000), n_families=3000,
                        length_dist=("lognormal", 300, 0.5, 30, 2500), core_frac=0.25,
                        accessory_draw=None, subst_max=0.30, indel_max=0.05, paralog_frac=0.10,
                        singleton_frac=0.05, seed=7),
    # Nucleotide stand-in: 8 genomes x Poisson(600) genes, gene lengths
    # log-normal with median 900 nt (300 codons), clipped to 90..7500, ACGT at
    # 50% GC, the pan50x3000 mutation model.
    "nt8x600": dict(n_genomes=8, genes_per_genome=("poisson", 600), n_families=800,
                    length_dist=("lognormal", 900, 0.5, 90, 7500), core_frac=0.4, accessory_draw=None,
                    subst_max=0.30, indel_max=0.05, paralog_frac=0.10, singleton_frac=0.05, seed=6,
                    alphabet="nt"),
}


# ---------------------------------------------------------------------------
# batches of independent genome-pair jobs
# ---------------------------------------------------------------------------

def _job_params(rng, n_jobs, genes=(500, 6000)):
    """Per-job generator parameters of a batch: gene counts U[genes] per
    genome (default U[500, 6000]), half of the jobs with log-normal lengths of median 300 aa and half
    with median 900 aa, and the pan50x3000 mutation model; families scale with
    the larger genome (4000 families per 3000 genes)."""
    m = rng.integers(genes[0], genes[1] + 1, size=(n_jobs, 2))
    long_len = np.zeros(n_jobs, dtype=bool)
    long_len[rng.permutation(n_jobs)[: n_jobs // 2]] = True
    seeds = rng.integers(0, 2**62, size=n_jobs)
    out = []
    for j in range(n_jobs):
        median = 900 if long_len[j] else 300
        out.append(dict(n_genomes=2, genes_per_genome=("list", [int(m[j, 0]), int(m[j, 1])]),
                        n_families=int(np.ceil(int(m[j].max()) * 4 / 3)),
                        length_dist=("lognormal", median, 0.5, 30, 2500), core_frac=0.4, accessory_draw=None,
                        subst_max=0.30, indel_max=0.05, paralog_frac=0.10, singleton_frac=0.05,
                        seed=int(seeds[j]), name=f"job{j}"))
    return out


def _generate_job(params):
    return generate(**params)


def concat(parts) -> Pangenome:
    """Datasets one after the other (genome i of part p keeps its order)."""
    res, gptr, gnm, fam = [], [np.zeros(1, np.int64)], [np.zeros(1, np.int64)], []
    r0, g0 = 0, 0
    for d in parts:
        res.append(d.residues)
        gptr.append(d.gene_ptr[1:] + r0)
        gnm.append(d.genome_ptr[1:].astype(np.int64) + g0)
        fam.append(d.family)
        r0 += d.n_residues
        g0 += d.n_genes
    return Pangenome(
        residues=np.concatenate(res) if res else np.zeros(0, np.uint8),
        gene_ptr=np.concatenate(gptr).astype(np.int64),
        genome_ptr=np.concatenate(gnm).astype(np.int32),
        family=np.concatenate(fam) if fam else np.zeros(0, np.int32),
        name="+".join(d.name for d in parts[:3]) + ("..." if len(parts) > 3 else ""),
    )


def job_batch(n_jobs: int = 2000, seed: int = 4, workers: int = 1, genes=(500, 6000)):
    """A batch of independent genome-pair jobs: returns (dataset, jobs) where
    job j compares genomes jobs[j, 0] = 2j and jobs[j, 1] = 2j+1 of the
    dataset.  Each job is its own two-genome pangenome (own families) drawn
    with the parameters of ``_job_params``; ``workers`` > 1 draws jobs in
    parallel processes (spawned, so it is safe after CUDA initialisation).
    ``genes`` is the range of genes per genome (smaller for quick tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = _job_params(rng, n_jobs, genes)
    if workers > 1 and n_jobs > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.map(_generate_job, params, chunksize=max(1, n_jobs // (4 * workers)))
    else:
        parts = [_generate_job(p) for p in params]
    ds = concat(parts)
    ds.name = f"jobs{n_jobs}"
    ds.params = dict(n_jobs=n_jobs, seed=seed)
    jobs = np.stack([np.arange(0, 2 * n_jobs, 2), np.arange(1, 2 * n_jobs, 2)], axis=1).astype(np.uint32)
    return ds, jobs


# ---------------------------------------------------------------------------
# a resident pangenome and a stream of incoming genomes
# ---------------------------------------------------------------------------

def served_stream(n_resident: int = 100, n_incoming: int = 500, seed: int = 5, resident_genes=("poisson", 3000),
                  incoming_genes=(1000, 7000), n_families: int = 4000) -> Pangenome:
    """One pangenome of n_resident + n_incoming genomes drawn from shared
    families with the pan50x3000 model: the first n_resident genomes (gene
    counts Poisson(3000) by default) form the resident set, the others (gene
    counts U[incoming_genes]) arrive one by one."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if resident_genes[0] == "poisson":
        res_counts = rng.poisson(resident_genes[1], size=n_resident)
    else:
        res_counts = rng.integers(resident_genes[1], resident_genes[2] + 1, size=n_resident)
    inc_counts = rng.integers(incoming_genes[0], incoming_genes[1] + 1, size=n_incoming)
    counts = [int(x) for x in np.concatenate([res_counts, inc_counts])]
    ds = generate(n_genomes=n_resident + n_incoming, genes_per_genome=("list", counts), n_families=n_families,
                  length_dist=("lognormal", 300, 0.5, 30, 2500), core_frac=0.4, accessory_draw=None,
                  subst_max=0.30, indel_max=0.05, paralog_frac=0.10, singleton_frac=0.05,
                  seed=int(rng.integers(0, 2**62)), name=f"served{n_resident}+{n_incoming}")
    ds.params.update(n_resident=n_resident, n_incoming=n_incoming)
    return ds


def genome_of(ds: Pangenome, i: int):
    """(residues, gene_ptr) of genome i alone."""
    g0, g1 = int(ds.genome_ptr[i]), int(ds.genome_ptr[i + 1])
    r0, r1 = int(ds.gene_ptr[g0]), int(ds.gene_ptr[g1])
    return ds.residues[r0:r1].copy(), (ds.gene_ptr[g0:g1 + 1] - r0).astype(np.int64)


def workload(name: str, **overrides) -> Pangenome:
    """Generate a named workload; keyword overrides replace model parameters."""
    params = dict(WORKLOADS[name])
    params.update(overrides)
    return generate(name=name, **params)


def random_tiny(seed: int, n_genomes: int = 3, max_genes: int = 6, max_len: int = 40,
                letters: bytes = ALPHABET) -> Pangenome:
    """Tiny random datasets over a letter subset (for brute-force checks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lets = np.frombuffer(letters, dtype=np.uint8)
    genomes = []
    for _ in range(n_genomes):
        m = int(rng.integers(1, max_genes + 1))
        genes = []
        for _ in range(m):
            L = int(rng.integers(0, max_len + 1))
            genes.append(lets[rng.integers(0, len(lets), size=L)].tobytes())
        genomes.append(genes)
    return from_strings(genomes)
