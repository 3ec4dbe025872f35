"""Helpers shared by the GPU parity tests: run both sides on one dataset and
put their outputs in the same shape (test infrastructure)."""
import numpy as np

import oracle
from paper_2510_23679_gb300 import pd, synth

LETTERS = synth.ALPHABET


def decode_code(code: int, k: int) -> bytes:
    """Base-20 code (first letter most significant) back to the k-mer string."""
    out = bytearray(k)
    for t in range(k - 1, -1, -1):
        out[t] = LETTERS[code % 20]
        code //= 20
    return bytes(out)


class DeviceRun:
    """One dataset profiled on the GPU (device handles kept for queries)."""

    def __init__(self, ctx, ds, k, device_inputs=False):
        import torch
        self.ctx, self.ds, self.k = ctx, ds, k
        res, gp, gn = ds.residues, ds.gene_ptr, ds.genome_ptr
        if device_inputs:
            res = torch.from_numpy(res).cuda() if res.size else torch.zeros(0, dtype=torch.uint8, device="cuda")
            gp = torch.from_numpy(gp).cuda()
            gn = torch.from_numpy(gn).cuda()
        self.prof = pd.pd_build_profiles(ctx, res, gp, gn, k)
        self.info = pd.pd_profiles_get_info(self.prof)

    def mv(self):
        mv_ptr, codes, counts, La = pd.pd_profiles_copy_mv(self.ctx, self.prof)
        out = []
        for g in range(self.ds.n_genes):
            e0, e1 = mv_ptr[g], mv_ptr[g + 1]
            out.append(([decode_code(int(c), self.k) for c in codes[e0:e1]], counts[e0:e1].tolist()))
        return out, La

    def summin(self, gi, gj):
        a, b, s = pd.pd_summin_pairs(self.ctx, self.prof, gi, gj)
        return {(int(x), int(y)): int(z) for x, y, z in zip(a, b, s)}

    def best_hits(self, gi, gj):
        h = pd.pd_best_hits(self.ctx, self.prof, gi, gj)
        rp, cols, s = pd.pd_hits_copy(self.ctx, h)
        return [cols[rp[x]:rp[x + 1]].tolist() for x in range(len(rp) - 1)], \
               [s[rp[x]:rp[x + 1]].tolist() for x in range(len(rp) - 1)]

    def bbh(self, gi, gj):
        return [tuple(x) for x in pd.pd_bbh_copy(self.ctx, pd.pd_bbh(self.ctx, self.prof, gi, gj)).tolist()]

    def all_pairs(self):
        hits = pd.pd_best_hits_all(self.ctx, self.prof)
        rp, cols, s = pd.pd_hits_copy(self.ctx, hits)
        bbh = pd.pd_bbh_copy(self.ctx, pd.pd_bbh_all(self.ctx, self.prof, hits))
        return rp, cols, s, bbh, pd.pd_hits_get_info(hits)


def oracle_pairs(ds, k, pairs, n_threads=1):
    """Oracle PairResult for each (gi, gj) (only those genomes are profiled)."""
    return {(gi, gj): oracle.pair_for_dataset(ds, gi, gj, k, n_threads) for gi, gj in pairs}


def oracle_nonzero(R):
    a, b = np.nonzero(R.S)
    return {(int(x), int(y)): int(R.S[x, y]) for x, y in zip(a, b)}


def csr_lists(ptr, idx):
    return [idx[ptr[x]:ptr[x + 1]].tolist() for x in range(len(ptr) - 1)]


def all_pairs_row_slice(ds, rp, cols, a_global, gj):
    """Best Hits of global gene a towards genome gj, as local indices in gj."""
    g0, g1 = int(ds.genome_ptr[gj]), int(ds.genome_ptr[gj + 1])
    row = cols[rp[a_global]:rp[a_global + 1]]
    return [int(b) - g0 for b in row if g0 <= b < g1]
