"""Benchmark: all-against-all gene similarity, Best Hits and BBH on one GB300.

One step = the whole hot path over one seeded synthetic pangenome: k-mer
profiles (encode, dictionary, multiplicity vectors, inverted index), sum-min
of every cross-genome gene pair sharing a k-mer, Best Hits of every gene in
every other genome, and Bidirectional Best Hits of every genome pair.

Prints one JSON line.  `value` is logical gene pairs (sum_{i<j} |G_i||G_j|)
per second with inputs resident in HBM; `e2e` is the same metric through the
public C ABI from pinned host buffers (host->device copy of the residues and
offsets and device->host copy of the BBH pairs inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload pan200x4000]
  python bench.py --impl reference ...   (the CPU oracle on bounded samples)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2510_23679_gb300 import synth  # noqa: E402

L2_FLUSH_BYTES = 512 << 20  # larger than the 129 MB L2
L2_NOTE = f"flushed ({L2_FLUSH_BYTES >> 20} MB write) between steps"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pan200x4000", choices=sorted(synth.WORKLOADS) + ["jobs", "served", "pairs"],
                    help="a plain pangenome, 'jobs': a batch of independent genome-pair jobs, or 'served': "
                         "genomes arriving at a resident index")
    ap.add_argument("--rates", default="2,5,10,20,50", help="arrival rates (genomes/s) of --workload served")
    ap.add_argument("--seconds-per-rate", type=float, default=20.0,
                    help="arrivals per rate: min(incoming, rate x this)")
    ap.add_argument("--incoming", type=int, default=500, help="incoming genomes of --workload served")
    ap.add_argument("--min-arrivals", type=int, default=100,
                    help="arrivals per rate of --workload served at least (so p99 is a percentile of many)")
    ap.add_argument("--pairs-of", default="pan200x4000", choices=sorted(synth.WORKLOADS),
                    help="the pangenome whose genome pairs --workload pairs compares")
    ap.add_argument("--jobs", type=int, default=2000, help="jobs in the batch (--workload jobs)")
    ap.add_argument("--no-per-pair", action="store_true", help="skip the one-pair-per-launch comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--walk", default="auto", choices=["auto", "merge", "warp"],
                    help="posting walk of the sum-min kernel (pd_ctx_set_walk); same results")
    ap.add_argument("--no-served", action="store_true",
                    help="skip the genome-add latency probe of the plain workload's line")
    ap.add_argument("--served-rate", type=float, default=20.0,
                    help="arrival rate (genomes/s) of the latency probe in the plain workload's line")
    ap.add_argument("--served-arrivals", type=int, default=100,
                    help="arrivals of the latency probe in the plain workload's line")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="bounded oracle sample length")
    ap.add_argument("--multi", default="shard", choices=["shard", "replicas"],
                    help="N > 1: 'shard' splits the one dataset's query genes across the ranks (the index is "
                         "replicated, the Best Hit rows are gathered to rank 0, BBH runs there); 'replicas' gives "
                         "each rank a dataset of its own")
    return ap.parse_args()


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x, world):
    """The largest x over all ranks (the slowest rank's time)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    if world == 1:
        return int(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([int(x)], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


def whole_job_rate(units, seconds, world):
    """Units processed by all ranks together / the slowest rank's time."""
    return sum_over_ranks(units, world) / max_over_ranks(seconds, world)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def make_workload(name, rank):
    ds = synth.workload(name) if rank == 0 else synth.workload(name, seed=synth.WORKLOADS[name]["seed"] + 1000 * rank)
    return ds


def parallelism_of(world, multi):
    if world == 1:
        return "1 GPU"
    if multi == "shard":
        return f"query genes sharded x{world}; index replicated; rows gathered to rank 0"
    return f"replicas x{world} (a dataset per rank)"


def config_of(ds, name, k, flush, parallelism="1 GPU"):
    return {"workload": f"{name}: {ds.n_genomes} genomes, {ds.n_genes} genes, {ds.n_residues} residues, "
                        f"k={k}, {'nucleotide' if alphabet_of(name) == 4 else 'amino-acid'} alphabet, "
                        f"all {ds.n_genomes * (ds.n_genomes - 1) // 2} genome pairs",
            "n_genomes": ds.n_genomes, "n_genes": ds.n_genes, "n_residues": ds.n_residues, "k": k,
            "logical_pairs_per_step": ds.logical_pairs(), "l2": flush, "parallelism": parallelism}


# --------------------------------------------------------------------------- CPU oracle sample
def captured_counter(kernel_src, summary, key="dram_bytes_per_launch"):
    """A per-launch counter (DRAM bytes by default) from the committed ncu
    summary of the dominant kernel on this workload, or None when there is no
    capture of it or the kernel source changed since."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
        sha = hashlib.sha256(open(os.path.join(ROOT, kernel_src), "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    m_sha = re.search(r"sha256 \(first 16 hex\): ([0-9a-f]{16})", text)
    m_val = re.search(re.escape(key) + r": (\d+)", text)
    if not m_sha or not m_val or m_sha.group(1) != sha:
        return None
    return int(m_val.group(1))


def alphabet_of(name):
    return 4 if synth.WORKLOADS.get(name, {}).get("alphabet") == "nt" else 20


def oracle_sample(ds, k, seconds, threads, alphabet=20):
    """Time the oracle (as it stands) on whole genome pairs until `seconds` pass."""
    import oracle
    n = ds.n_genomes
    pairs = [(i, i + 1) for i in range(0, n - 1, 2)]
    done, pairs_done, t0 = [], 0, time.perf_counter()
    for gi, gj in pairs:
        oracle.pair_for_dataset(ds, gi, gj, k, n_threads=threads, alphabet=alphabet)
        done.append((gi, gj))
        pairs_done += int(ds.genome_ptr[gi + 1] - ds.genome_ptr[gi]) * int(ds.genome_ptr[gj + 1] - ds.genome_ptr[gj])
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return pairs_done / dt, dt, done, pairs_done


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        # samples of this process only, summarised into the JSON line
        self.path = os.path.join(tempfile.gettempdir(), f"pd_clocks_{os.getpid()}_{device_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    ds = make_workload(args.workload, 0)
    import oracle
    alpha = alphabet_of(args.workload)
    k = oracle.choose_k(ds.n_residues, alphabet=alpha)
    cores = host_cores()
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps))
    for _ in range(args.warmup):
        oracle_sample(ds, k, 0.0, cores, alpha)  # one genome pair each
    rates, samples, step_ms = [], [], []
    for _ in range(args.steps):
        r, dt, done, npairs = oracle_sample(ds, k, per_step, cores, alpha)
        rates.append(r)
        samples.append(npairs)
        step_ms.append(dt * 1e3)
    value = statistics.median(rates)
    # ms_per_step is the measured time of one sampled step; the time the
    # oracle would take for the whole workload is extrapolated from its rate
    line = {"metric": "gene-pair GJ evals/s", "value": value, "unit": "gene-pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(step_ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "impl": "reference",
            "config": config_of(ds, args.workload, k, L2_NOTE, parallelism_of(world, args.multi)),
            "step": "a bounded sample of the workload: whole genome pairs until the per-step time is reached",
            "whole_workload_ms_extrapolated": ds.logical_pairs() / value * 1e3,
            "cpu_baseline": {"value": value, "unit": "gene-pairs/s", "cores": cores, "kind": "oracle",
                             "sample": f"whole genome pairs of the workload per step (~{per_step:.0f} s each, "
                                       f"{statistics.median(samples):.3g} gene pairs), oracle threads={cores}"},
            "e2e": {"value": value, "unit": "gene-pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- our arm
# --------------------------------------------------------------------------- batched jobs
def run_batch(args):
    """Batched form: n genome-pair jobs (gene counts U[500, 6000], half of the
    jobs with median gene length 300 aa and half 900 aa), each at its own k,
    through pd_bbh_batch, next to the same jobs run one pair per launch
    sequence (pd_build_profiles + pd_best_hits_all + pd_bbh_all on each job's
    two genomes).  Both produce every Best Hit of both directions and every
    BBH pair of every job."""
    cores = host_cores()
    t0 = time.perf_counter()
    ds, jobs = synth.job_batch(args.jobs, seed=4, workers=min(cores, 32))
    gen_s = time.perf_counter() - t0
    import torch
    from paper_2510_23679_gb300 import pd
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gp, gnm = ds.gene_ptr, ds.genome_ptr
    sizes = np.diff(gnm).astype(np.int64)
    n_res_job = [int(gp[gnm[b + 1]] - gp[gnm[a]]) for a, b in jobs]
    ks = np.array([pd.pd_choose_k(n) for n in n_res_job], np.int32)
    pairs = int(sum(sizes[a] * sizes[b] for a, b in jobs))
    ctx = pd.pd_ctx_create(local)
    stream = torch.cuda.current_stream(dev)
    res_d = torch.from_numpy(ds.residues).to(dev)
    gp_d = torch.from_numpy(gp).to(dev)
    gn_d = torch.from_numpy(gnm).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    # autotune on a sample of the jobs, then run the whole batch with the winner
    t_tune = time.perf_counter()
    tuning, tune_ms_per_job = pd.pd_batch_autotune(ctx, res_d, gp_d, gn_d, jobs, ks, n_sample=min(100, args.jobs))
    tune_s = time.perf_counter() - t_tune

    def step_batch():
        return pd.pd_bbh_batch(ctx, res_d, gp_d, gn_d, jobs, ks, **tuning)

    for _ in range(args.warmup):
        step_batch()
    torch.cuda.synchronize()
    launches0 = pd.pd_ctx_launch_count(ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    keep = None
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(i)
            ev[i][0].record(stream)
            keep = step_batch()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    gpu_launches = pd.pd_ctx_launch_count(ctx) - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    info = pd.pd_batch_get_info(keep)

    per_pair = None
    if not args.no_per_pair:
        views = []
        for (a, b) in jobs:
            g0, g1 = int(gnm[a]), int(gnm[b + 1])
            r0, r1 = int(gp[g0]), int(gp[g1])
            views.append((res_d[r0:r1], (gp_d[g0:g1 + 1] - r0).contiguous(),
                          torch.tensor([0, int(sizes[a]), int(sizes[a] + sizes[b])], dtype=torch.int32, device=dev)))

        def step_pairs():
            n = 0
            for (r, g, gn), k in zip(views, ks):
                p = pd.pd_build_profiles(ctx, r, g, gn, int(k))
                h = pd.pd_best_hits_all(ctx, p)
                n += pd.pd_bbh_count(pd.pd_bbh_all(ctx, p, h))
            return n

        step_pairs()
        torch.cuda.synchronize()
        flush.fill_(7)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n_pp = step_pairs()
        e1.record(stream)
        torch.cuda.synchronize()
        pp_ms = e0.elapsed_time(e1)
        assert n_pp == info.n_bbh, (n_pp, info.n_bbh)
        per_pair = {"ms_per_step": pp_ms, "value": pairs / (pp_ms / 1e3), "unit": "gene-pairs/s",
                    "steps": 1, "bbh_pairs": n_pp}

    value = whole_job_rate(pairs, ms / 1e3, world)
    jobs_rate = whole_job_rate(args.jobs, ms / 1e3, world)
    ms = max_over_ranks(ms, world)
    if rank == 0:
        line = {
            "metric": "gene-pair GJ evals/s", "value": value, "unit": "gene-pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "impl": "batched",
            "config": {"workload": f"jobs{args.jobs}: {args.jobs} genome-pair jobs, {ds.n_genes} genes, "
                                   f"{ds.n_residues} residues, k per job by the residue rule",
                       "k_counts": {int(k): int(c) for k, c in zip(*np.unique(ks, return_counts=True))},
                       "n_jobs": args.jobs, "n_genes": ds.n_genes, "n_residues": ds.n_residues,
                       "logical_pairs_per_step": pairs, "l2": "flushed between steps",
                       "generation_s": gen_s},
            "genome_pairs_per_s": jobs_rate,
            "step_ms": step_ms,
            "tuning": tuning, "autotune": {"sample_jobs": min(100, args.jobs), "seconds": tune_s,
                                            "best_ms_per_sampled_job": tune_ms_per_job},
            "per_pair_launch": per_pair,
            "speedup_vs_per_pair": (per_pair["ms_per_step"] / ms) if per_pair else None,
            "gpu_launches": gpu_launches,
            "clocks": clk.summary(),
            "stats": {"chunks": info.n_chunks, "best_hits": info.n_hits, "bbh_pairs": info.n_bbh,
                      "postings_walked": info.postings_walked},
        }
        print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- served index
def serve_rate(pd, ctx, res, k, incoming, rate, n, budget, rng):
    """Serve the first n incoming genomes, arriving as a Poisson process of
    `rate` genomes/s, on a fresh index over the resident pangenome `res`.
    Latency = answer time - submission time (the library's steady clock)."""
    gaps = rng.exponential(1.0 / rate, size=n)
    index = pd.pd_index_create(ctx, res.residues, res.gene_ptr, res.genome_ptr, k, budget)
    # warm-up: one request through a separate index of the same size
    warm = pd.pd_index_create(ctx, res.residues, res.gene_ptr, res.genome_ptr, k, budget)
    pd.pd_index_poll(warm, pd.pd_index_submit(warm, *incoming[0]), -1)
    warm.free()
    tickets = []
    start = time.perf_counter()
    due = start
    for i in range(n):
        due += gaps[i]
        d = due - time.perf_counter()
        if d > 0:
            time.sleep(d)
        tickets.append(pd.pd_index_submit(index, *incoming[i]))
    lat, wait, service, t_first, t_last, ticks = [], [], [], None, None, []
    for t in tickets:
        info = pd.pd_reply_get_info(pd.pd_index_poll(index, t, -1))
        assert info.status == 0, info.status
        lat.append((info.t_done_ns - info.t_submit_ns) / 1e6)
        wait.append((info.t_start_ns - info.t_submit_ns) / 1e6)
        service.append((info.t_done_ns - info.t_start_ns) / 1e6)
        t_first = info.t_submit_ns if t_first is None else min(t_first, info.t_submit_ns)
        t_last = info.t_done_ns if t_last is None else max(t_last, info.t_done_ns)
        ticks.append(info.tick_requests)
    ii = pd.pd_index_get_info(index)
    out = {"arrivals": n, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "mean_ms": float(np.mean(lat)), "max_ms": float(np.max(lat)),
           "queue_wait_p50_ms": float(np.percentile(wait, 50)), "queue_wait_p99_ms": float(np.percentile(wait, 99)),
           "tick_p50_ms": float(np.percentile(service, 50)), "tick_p99_ms": float(np.percentile(service, 99)),
           "sustained_genomes_per_s": n / ((t_last - t_first) / 1e9),
           "offered_genomes_per_s": rate, "ticks": int(ii.ticks),
           "max_requests_per_tick": int(ii.max_tick_requests),
           "resident_genomes_at_end": int(ii.n_genomes),
           "index_device_bytes_at_end": int(ii.device_bytes)}
    index.free()
    return out


def served_probe(args, pd, ctx):
    """Genome-add latency beside the plain workload's throughput: a resident
    index of 100 genomes of the pan50x3000 model answers `served_arrivals`
    incoming genomes (U[1000, 7000] genes) arriving at `served_rate`/s."""
    t0 = time.perf_counter()
    ds = synth.served_stream(100, args.served_arrivals, seed=5)
    gen_s = time.perf_counter() - t0
    res = ds.subset(list(range(100)))
    k = pd.pd_choose_k(res.n_residues)
    incoming = [synth.genome_of(ds, x) for x in range(100, ds.n_genomes)]
    rng = np.random.Generator(np.random.PCG64(55))
    out = serve_rate(pd, ctx, res, k, incoming, args.served_rate, len(incoming), 120 << 30, rng)
    out.update({"resident_genomes": 100, "resident_genes": res.n_genes, "k": k, "hbm_budget_bytes": 120 << 30,
                "generation_s": gen_s,
                "workload": f"resident 100 genomes (pan50x3000 model, {res.n_genes} genes, k={k}); "
                            f"{len(incoming)} incoming genomes of U[1000,7000] genes, Poisson arrivals at "
                            f"{args.served_rate:g}/s"})
    return out


def run_served(args):
    """Served form: a resident index of 100 genomes (the pan50x3000 model)
    answers incoming genomes (gene counts U[1000, 7000]) arriving as a
    Poisson process; each answer holds the genome's Best Hits in every
    resident genome and its BBH pairs, after which the genome is resident.
    For each arrival rate a fresh index serves min(incoming, max(min-arrivals,
    rate x seconds-per-rate)) arrivals; latency = answer time - submission time (the
    library's steady clock).  Beside it: one full recomputation (profiles,
    all-pairs Best Hits and BBH of every genome) at the final size."""
    t0 = time.perf_counter()
    ds = synth.served_stream(100, args.incoming, seed=5)
    gen_s = time.perf_counter() - t0
    import torch
    from paper_2510_23679_gb300 import pd
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n_res = 100
    res = ds.subset(list(range(n_res)))
    k = pd.pd_choose_k(res.n_residues)
    ctx = pd.pd_ctx_create(0)
    budget = 120 << 30
    incoming = [synth.genome_of(ds, x) for x in range(n_res, ds.n_genomes)]
    rng = np.random.Generator(np.random.PCG64(55))
    per_rate = {}
    clk_all = None
    with ClockSampler(0) as clk:
        for rate in [float(x) for x in args.rates.split(",")]:
            n = int(min(len(incoming), max(args.min_arrivals, round(rate * args.seconds_per_rate))))
            per_rate[str(rate)] = serve_rate(pd, ctx, res, k, incoming, rate, n, budget, rng)
            torch.cuda.synchronize()
        clk_all = clk.summary()
    # full recomputation at the final size (every genome, all pairs)
    n_last = 100 + max(v["arrivals"] for v in per_rate.values())
    full = ds.subset(list(range(n_last)))
    r_d = torch.from_numpy(full.residues).to(dev)
    g_d = torch.from_numpy(full.gene_ptr).to(dev)
    n_d = torch.from_numpy(full.genome_ptr).to(dev)

    def recompute():
        p = pd.pd_build_profiles(ctx, r_d, g_d, n_d, k)
        h = pd.pd_best_hits_all(ctx, p)
        return pd.pd_bbh_count(pd.pd_bbh_all(ctx, p, h))

    recompute()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    recompute()
    e1.record()
    torch.cuda.synchronize()
    full_ms = e0.elapsed_time(e1)
    top = per_rate[max(per_rate, key=lambda r: float(r))]
    line = {"metric": "p50/p99 genome-add latency; sustained genomes/s", "value": top["sustained_genomes_per_s"],
            "unit": "genomes/s", "n_gpus": 1, "steps": len(per_rate), "warmup": 1,
            "ms_per_step": top["mean_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic", "impl": "served",
            "config": {"workload": f"served: resident 100 genomes ({res.n_genes} genes, k={k}), "
                                   f"{args.incoming} incoming genomes of U[1000,7000] genes, Poisson arrivals",
                       "hbm_budget_bytes": budget, "generation_s": gen_s},
            "latency_by_rate": per_rate,
            "recompute_all": {"genomes": n_last, "ms": full_ms, "genomes_per_s_if_recomputed_per_arrival":
                              1e3 / full_ms},
            "clocks": clk_all}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- genome pairs of one dataset
def run_pairs(args):
    """pd_bbh_pairs on --jobs random genome pairs of one profiled pangenome
    (--pairs-of, default pan200x4000), next to the same pairs one pd_bbh call
    each (its BBH only: the one-pair path's least work)."""
    import torch
    from paper_2510_23679_gb300 import pd
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ds = synth.workload(args.pairs_of)
    k = pd.pd_choose_k(ds.n_residues)
    ctx = pd.pd_ctx_create(0)
    prof = pd.pd_build_profiles(ctx, torch.from_numpy(ds.residues).to(dev), torch.from_numpy(ds.gene_ptr).to(dev),
                                torch.from_numpy(ds.genome_ptr).to(dev), k)
    rng = np.random.default_rng(12)
    jobs = []
    while len(jobs) < args.jobs:
        a, b = rng.integers(0, ds.n_genomes, size=2)
        if a != b:
            jobs.append((int(a), int(b)))
    jobs = np.array(jobs, np.uint32)
    sizes = np.diff(ds.genome_ptr).astype(np.int64)
    pairs = int(sum(sizes[a] * sizes[b] for a, b in jobs))
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        out = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return sorted(out)[len(out) // 2], r

    def batched():
        return pd.pd_batch_get_info(pd.pd_bbh_pairs(ctx, prof, jobs)).n_bbh

    def one_by_one():
        return sum(pd.pd_bbh_count(pd.pd_bbh(ctx, prof, int(a), int(b))) for a, b in jobs)

    for _ in range(args.warmup):
        batched()
    one_by_one()
    with ClockSampler(0) as clk:
        ms_b, n_b = timed(batched, args.steps)
        ms_1, n_1 = timed(one_by_one, 1)
    assert n_b == n_1, (n_b, n_1)
    print(json.dumps({
        "metric": "gene-pair GJ evals/s", "value": pairs / (ms_b / 1e3), "unit": "gene-pairs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic", "impl": "pairs",
        "config": {"workload": f"{args.jobs} random genome pairs of {args.pairs_of} (k={k}), profiles resident",
                   "logical_pairs_per_step": pairs},
        "genome_pairs_per_s": args.jobs / (ms_b / 1e3),
        "one_pair_per_call": {"ms": ms_1, "genome_pairs_per_s": args.jobs / (ms_1 / 1e3)},
        "speedup_vs_one_pair_per_call": ms_1 / ms_b, "bbh_pairs": n_b, "clocks": clk.summary()}))
    return 0


# --------------------------------------------------------------------------- one dataset over N GPUs
def run_sharded(args):
    """N > 1, one dataset: every rank profiles the whole dataset (the index is
    replicated), computes the Best Hit rows of its shard of the query genes
    (pd_best_hits_shard), the rows are all-gathered (NCCL) and rank 0
    assembles them (pd_hits_import) and runs BBH.  value = the dataset's
    logical pairs / the slowest rank's step time (strong scaling)."""
    import torch
    import torch.distributed as dist
    from paper_2510_23679_gb300 import pd, shards
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    ds = synth.workload(args.workload)
    alpha = alphabet_of(args.workload)
    k = pd.pd_choose_k(ds.n_residues, alpha)
    ctx = pd.pd_ctx_create(local)
    stream = torch.cuda.current_stream(dev)
    res_d = torch.from_numpy(ds.residues).to(dev)
    gp_d = torch.from_numpy(ds.gene_ptr).to(dev)
    gn_d = torch.from_numpy(ds.genome_ptr).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def step(res, gp, gn):
        prof = pd.pd_build_profiles_alphabet(ctx, res, gp, gn, alpha, k)
        hits, bbh = shards.sharded_bbh(ctx, prof)
        return prof, hits, bbh

    for _ in range(args.warmup):
        step(res_d, gp_d, gn_d)
    torch.cuda.synchronize()
    pd.pd_ctx_reset_timing(ctx)
    pd.pd_ctx_set_timing_filter(ctx, "summin_bh")
    pd.pd_ctx_set_timing(ctx, True)
    launches0 = pd.pd_ctx_launch_count(ctx)
    times = []
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(i)
            dist.barrier()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            keep = step(res_d, gp_d, gn_d)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    dist.barrier()
    gpu_launches = pd.pd_ctx_launch_count(ctx) - launches0
    k_ms, k_n = pd.pd_ctx_kernel_time(ctx, "summin_bh")
    pd.pd_ctx_set_timing(ctx, False)
    ms_local = sum(times) / len(times)
    ms = max_over_ranks(ms_local, world)
    pairs = ds.logical_pairs()
    # roofline of this rank's shard: its postings walked and hits, and its
    # share (1/world) of the vector, row and gene bytes
    prof, hits, bbh = keep
    pinfo = pd.pd_profiles_get_info(prof)
    shard_hits = pd.pd_hits_get_info(pd.pd_best_hits_shard(ctx, prof, rank, world))
    alg = (pinfo.n_entries * 14 + pinfo.n_genes * 12) / world + shard_hits.postings_walked * 4 + \
        shard_hits.n_hits * 8
    k_avg = k_ms / max(1, k_n)
    peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    clocks = clk.summary()
    if rank == 0:
        line = {"metric": "gene-pair GJ evals/s", "value": pairs / (ms / 1e3), "unit": "gene-pairs/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic",
                "config": config_of(ds, args.workload, k, L2_NOTE, parallelism_of(world, "shard")),
                "genome_pairs_per_s": ds.n_genomes * (ds.n_genomes - 1) // 2 / (ms / 1e3), "step_ms": times,
                "roofline": {"bound": "hbm", "achieved": alg / (k_avg / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                             "frac": alg / (k_avg / 1e3) / 1e9 / peak, "traffic": None, "kernel": "summin_bh",
                             "kernel_ms": k_avg, "alg_bytes": alg, "scope": "rank 0's shard"},
                "e2e": None, "gpu_launches": gpu_launches, "cpu_baseline": None, "clocks": clocks,
                "stats": {"best_hits": pd.pd_hits_get_info(hits).n_hits, "bbh_pairs": pd.pd_bbh_count(bbh)}}
        print(json.dumps(line))
    dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "jobs":
        return run_batch(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "pairs":
        return run_pairs(args)
    import torch
    from paper_2510_23679_gb300 import pd

    rank, world, local = dist_info()
    if world > 1 and args.multi == "shard":
        return run_sharded(args)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ds = make_workload(args.workload, rank)
    alpha = alphabet_of(args.workload)
    k = pd.pd_choose_k(ds.n_residues, alpha)
    ctx = pd.pd_ctx_create(local)
    pd.pd_ctx_set_walk(ctx, {"auto": pd.PD_WALK_AUTO, "merge": pd.PD_WALK_MERGE, "warp": pd.PD_WALK_WARP}[args.walk])
    stream = torch.cuda.current_stream(dev)

    res_d = torch.from_numpy(ds.residues).to(dev)
    gp_d = torch.from_numpy(ds.gene_ptr).to(dev)
    gn_d = torch.from_numpy(ds.genome_ptr).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def step_device():
        prof = pd.pd_build_profiles_alphabet(ctx, res_d, gp_d, gn_d, alpha, k)
        hits = pd.pd_best_hits_all(ctx, prof)
        bbh = pd.pd_bbh_all(ctx, prof, hits)
        return prof, hits, bbh

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- device-resident timed region (per-launch events on the dominant
    # kernel only, so the other launches run without event records)
    pd.pd_ctx_reset_timing(ctx)
    pd.pd_ctx_set_timing_filter(ctx, "summin_bh")
    pd.pd_ctx_set_timing(ctx, True)
    launches0 = pd.pd_ctx_launch_count(ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    keep = None
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(i)  # evict the previous step's data from L2 (not timed)
            ev[i][0].record(stream)
            keep = step_device()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    barrier()
    gpu_launches = pd.pd_ctx_launch_count(ctx) - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    k_ms, k_n = pd.pd_ctx_kernel_time(ctx, "summin_bh")
    pd.pd_ctx_set_timing(ctx, False)
    pd.pd_ctx_set_timing_filter(ctx, None)
    ms_local = sum(step_ms) / len(step_ms)
    pairs = ds.logical_pairs()
    value = whole_job_rate(pairs, ms_local / 1e3, world)
    ms_per_step = max_over_ranks(ms_local, world)
    genome_pairs_all = sum_over_ranks(ds.n_genomes * (ds.n_genomes - 1) // 2, world)

    prof, hits, bbh = keep
    pinfo = pd.pd_profiles_get_info(prof)
    hinfo = pd.pd_hits_get_info(hits)
    n_bbh = pd.pd_bbh_count(bbh)

    # ---- roofline of the dominant kernel (sum-min + Best Hits), algorithmic bytes per launch
    E = pinfo.n_entries
    J = hinfo.postings_walked
    alg_bytes = E * 6 + E * 8 + J * 4 + hinfo.n_hits * 8 + pinfo.n_genes * 12
    k_avg_ms = k_ms / max(1, k_n)
    achieved = alg_bytes / (k_avg_ms / 1e3) / 1e9
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except (OSError, ValueError):
        pass  # no measured peaks on this machine: the recipe's fallback, labelled as such
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    # ---- per-phase breakdown, after the timed region: each phase's wall time
    # on the stream and the device time of its kernels (CUDA events around
    # every launch), medians of three L2-flushed steps
    def timed_phase(fn):
        pd.pd_ctx_reset_timing(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        kms, kn = pd.pd_ctx_kernel_time(ctx, None)  # synchronizes the stream
        return out, e0.elapsed_time(e1), kms, kn

    ph = {"build": [], "best_hits": [], "bbh": []}
    pd.pd_ctx_set_timing(ctx, True)
    for i in range(3):
        flush.fill_(i)
        torch.cuda.synchronize()
        p_, *t_b = timed_phase(lambda: pd.pd_build_profiles_alphabet(ctx, res_d, gp_d, gn_d, alpha, k))
        h_, *t_h = timed_phase(lambda: pd.pd_best_hits_all(ctx, p_))
        _, *t_x = timed_phase(lambda: pd.pd_bbh_all(ctx, p_, h_))
        for name, t in (("build", t_b), ("best_hits", t_h), ("bbh", t_x)):
            ph[name].append(t)
    pd.pd_ctx_set_timing(ctx, False)
    phases = {name: {"ms": statistics.median(t[0] for t in v), "kernel_ms": statistics.median(t[1] for t in v),
                     "launches": int(v[0][2])} for name, v in ph.items()}
    # encoder (profiles + inverted index) roofline: algorithmic bytes of one build
    W, D = pinfo.n_windows, pinfo.n_distinct
    passes = (max(1, int(D).bit_length()) + 8) // 9
    enc_bytes = (2 * ds.n_residues + E * 6 + pinfo.n_genes * 4 + W * 8 + passes * W * 16
                 + W * 8 + E * 4 + D * 4 + E * 12)
    enc_ms = phases["build"]["kernel_ms"]
    encoder = {"bound": "hbm", "alg_bytes": int(enc_bytes), "kernel_ms": enc_ms,
               "achieved": enc_bytes / (enc_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
               "frac": enc_bytes / (enc_ms / 1e3) / 1e9 / peak, "sort_passes": passes}

    # ---- the merge form of Eq. (5) (pd_summin_list: two sorted vectors
    # walked side by side, one warp per pair) on this step's BBH pairs, once
    merge_form = None
    if n_bbh:
        a_d, b_d = torch.empty(n_bbh, dtype=torch.int32, device=dev), torch.empty(n_bbh, dtype=torch.int32, device=dev)
        pd.pd_bbh_copy(ctx, bbh, a_d, b_d)
        s_d, den_d = torch.empty_like(a_d), torch.empty_like(a_d)
        for rep in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pd.pd_summin_list(ctx, prof, a_d, b_d, s_d, den_d)
            e1.record(stream)
            torch.cuda.synchronize()
        m_ms = e0.elapsed_time(e1)
        merge_form = {"pairs": n_bbh, "ms": m_ms, "pairs_per_s": n_bbh / (m_ms / 1e3),
                      "what": "sum-min and sum-max of every BBH pair of the step by the two-pointer merge of their "
                              "sorted multiplicity vectors (the vectors of the genes involved sorted first)"}
        del a_d, b_d, s_d, den_d

    # ---- end to end through the C ABI from pinned host buffers: inputs
    # copied in, and the whole result (the Best Hit CSR with each hit's
    # sum-min, and the BBH pairs) copied back, every step
    e2e = None
    if not args.no_e2e:
        res_h = torch.from_numpy(ds.residues).pin_memory()
        gp_h = torch.from_numpy(ds.gene_ptr).pin_memory()
        gn_h = torch.from_numpy(ds.genome_ptr).pin_memory()
        n_hits0 = int(hinfo.n_hits)
        host = {"a": torch.empty(max(n_bbh, 1), dtype=torch.int32).pin_memory(),
                "b": torch.empty(max(n_bbh, 1), dtype=torch.int32).pin_memory(),
                "row_ptr": torch.empty(ds.n_genes + 1, dtype=torch.int64).pin_memory(),
                "cols": torch.empty(max(n_hits0, 1), dtype=torch.int32).pin_memory(),
                "s": torch.empty(max(n_hits0, 1), dtype=torch.int32).pin_memory()}
        d2h = 0

        def fit(name, n, dtype):
            if n > host[name].numel():
                host[name] = torch.empty(n, dtype=dtype).pin_memory()
            return host[name]

        def step_e2e():
            nonlocal d2h
            p = pd.pd_build_profiles_alphabet(ctx, res_h, gp_h, gn_h, alpha, k)
            h = pd.pd_best_hits_all(ctx, p)
            b = pd.pd_bbh_all(ctx, p, h)
            nh = int(pd.pd_hits_get_info(h).n_hits)
            pd.pd_hits_copy(ctx, h, host["row_ptr"], fit("cols", nh, torch.int32), fit("s", nh, torch.int32))
            n = pd.pd_bbh_count(b)
            pd.pd_bbh_copy(ctx, b, fit("a", n, torch.int32), fit("b", n, torch.int32))
            d2h = 8 * n + 8 * (ds.n_genes + 1) + 8 * nh

        for _ in range(2):
            step_e2e()
        torch.cuda.synchronize()
        barrier()
        times = []
        for i in range(args.steps):
            flush.fill_(i)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_e2e()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        e2e_local = sum(times) / len(times)
        e2e_value = whole_job_rate(pairs, e2e_local, world)
        e2e_s = max_over_ranks(e2e_local, world)
        e2e = {"value": e2e_value, "unit": "gene-pairs/s",
               "h2d_bytes_per_step": int(ds.residues.nbytes + ds.gene_ptr.nbytes + ds.genome_ptr.nbytes),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3,
               "copied_back": "Best Hit CSR (row offsets, columns, sum-min) and BBH pairs"}

    served = None
    if rank == 0 and world == 1 and not args.no_served:
        served = served_probe(args, pd, ctx)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        rate, dt, done, npairs = oracle_sample(ds, k, args.cpu_seconds, cores, alpha)
        cpu = {"value": rate, "unit": "gene-pairs/s", "cores": cores, "kind": "oracle",
               "sample": f"genome pairs {done} of the same workload ({npairs} gene pairs, {dt:.1f} s, "
                         f"profiles of both genomes included), oracle threads={cores}"}

    # the pipe that bounds the sum-min kernel: L1TEX data-pipe wavefronts
    # (shared-memory accumulator + posting loads; ncu counts one launch) per
    # second of the live kernel time, against one wavefront per cycle per SM
    # at the SM clock sampled during the timed region
    clocks = clk.summary()
    wavefronts = captured_counter("paper_2510_23679_gb300/csrc/k_summin.cu", f"summin_bh_{args.workload}.md",
                                  "l1tex_wavefronts_per_launch")
    l1tex = None
    if wavefronts and clocks.get("sm_mhz"):
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        l1_peak = n_sm * clocks["sm_mhz"] * 1e6 / 1e9
        l1_achieved = wavefronts / (k_avg_ms / 1e3) / 1e9
        l1tex = {"bound": "l1tex", "kernel": "summin_bh", "achieved": l1_achieved, "peak": l1_peak,
                 "unit": "G wavefronts/s", "frac": l1_achieved / l1_peak, "wavefronts": wavefronts,
                 "peak_source": f"{n_sm} SMs x 1 wavefront/cycle x {clocks['sm_mhz']:.0f} MHz"}

    if rank == 0:
        line = {
            "metric": "gene-pair GJ evals/s", "value": value, "unit": "gene-pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": dict(config_of(ds, args.workload, k, L2_NOTE, parallelism_of(world, "replicas")),
                           **({} if args.walk == "auto" else {"walk": args.walk})),
            "genome_pairs_per_s": genome_pairs_all / (ms_per_step / 1e3),
            "step_ms": step_ms,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": captured_counter("paper_2510_23679_gb300/csrc/k_summin.cu",
                                                     f"summin_bh_{args.workload}.md"),
                         "kernel": "summin_bh",
                         "kernel_ms": k_avg_ms, "alg_bytes": alg_bytes, "peak_source": peak_src},
            "e2e": e2e,
            "served": served,
            "merge_form": merge_form,
            "phases": phases,
            "encoder_roofline": encoder,
            "l1tex_roofline": l1tex,
            "gpu_launches": gpu_launches,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "stats": {"n_distinct_kmers": pinfo.n_distinct, "mv_entries": E, "postings_walked": J,
                      "best_hits": hinfo.n_hits, "bbh_pairs": n_bbh, "deferred_queries": hinfo.n_deferred,
                      "max_posting": pinfo.max_posting, "profile_bytes": pinfo.device_bytes},
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
