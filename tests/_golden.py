"""Reader for the hand-worked fixtures in tests/golden/."""
import os
from dataclasses import dataclass, field

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@dataclass
class Golden:
    name: str
    k: int
    rows: list
    cols: list
    La_rows: list
    La_cols: list
    S: list          # [row][col] -> (s, sum_max)
    row_bh: list     # [row] -> list of cols
    col_bh: list     # [col] -> list of rows
    bbh: list        # [(a, b)]
    mv: dict = field(default_factory=dict)   # gene -> [(kmer, count)]


def _sets(txt):
    out = []
    for part in txt.split(";"):
        part = part.strip()
        out.append([] if part == "-" else [int(x) for x in part.split(",")])
    return out


def load(fname):
    kv, mv = {}, {}
    with open(os.path.join(GOLDEN_DIR, fname)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = [x.strip() for x in line.split("=", 1)]
            if key.startswith("mv "):
                mv[key[3:].strip()] = [(t.split(":")[0], int(t.split(":")[1])) for t in val.split()]
            else:
                kv[key] = val
    S = []
    for row in kv["S"].split(";"):
        S.append([tuple(int(x) for x in cell.split("/")) for cell in row.split()])
    bbh = [tuple(int(x) for x in t.split(":")) for t in kv["bbh"].split()]
    return Golden(name=fname, k=int(kv["k"]), rows=kv["rows"].split(), cols=kv["cols"].split(),
                  La_rows=[int(x) for x in kv["La_rows"].split()],
                  La_cols=[int(x) for x in kv["La_cols"].split()], S=S,
                  row_bh=_sets(kv["row_bh"]), col_bh=_sets(kv["col_bh"]), bbh=bbh, mv=mv)


def all_fixtures():
    return sorted(f for f in os.listdir(GOLDEN_DIR) if f.endswith(".txt"))
