"""Throughput of the LSHBloom deduplication path on one GB300 (or N replicas).

A step is one pass of the whole path over one batch: the peS2o-shaped batch
of 1,000,000 synthetic documents (lognormal median 3,000 tokens, Zipf(1.1)
over 200k words, 10% near-duplicates at Jaccard 0.6-0.95; 5-gram shingles,
P=121, b=11, r=11, filters sized for n=39M at p=1e-5), generated in HBM.
Each step clears the filters and deduplicates the whole batch, so every step
does the same work.

Prints one JSON line (rank 0).  `value` is docs/s of the batched form with
inputs resident in HBM; `plain` is the one-kernel-per-stage form on the same
batch; `e2e` is the same metric through lshbloom_dedup with pinned host
buffers, host<->device copies inside the timed region.  Beside them:
`roofline` (the persistent signature kernel against the integer-multiply
peak, and against the measured ceiling of its own arithmetic),
`roofline_probe` (the Bloom probe kernel against the copy peak and the
measured random-sector rates), `index_variants` (blocked filters, exact
band-key sets, weighted band keys), `serve`, `configs` (the 10k-document,
8M-document Pareto and billion-document configurations, each with its own
clocks and CPU baselines), `cpu_baseline` (the oracle, one thread, bounded
sample), `cpu_threaded` (the oracle on all host cores, the paper's CPU
design) and `device_peaks` (microbench/peaks.cu).

--impl reference times the CPU oracle (single thread) on a bounded sample of
the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (spec factory, n_docs, n_expected, fp_rate, tokens, shingles); the
    # token and shingle counts are those the generator gives rank 0 (checked)
    "pes2o_1m": ("pes2o_shaped", 1_000_000, 39_000_000, 1e-5, 4_917_430_137, 4_913_430_137),
    # the first 100k documents of the same corpus, same filters (still > L2): profiling case
    "pes2o_100k": ("pes2o_shaped", 100_000, 39_000_000, 1e-5, 489_419_695, 489_019_695),
    "plain_10k": ("plain_10k", 10_000, 10_000, 1e-5, 6_425_246, 6_385_246),
}
P, BANDS, ROWS, NGRAM = 121, 11, 11, 5
METRIC = "docs/s (LSHBloom dedup: shingle SHA-1, MinHash P=121, 11x11 bands, Bloom query+insert)"


def _config(name, world):
    """The workload as both arms report it."""
    _, D, nexp, fp, T, S = WORKLOADS[name]
    return {"workload": f"{name}: {D} docs, {T} tokens, {S} shingles", "P": P, "bands": BANDS,
            "rows": ROWS, "ngram": NGRAM, "n_expected": nexp, "fp_rate": fp,
            "l2": "inputs larger than L2 (tokens %.1f GB)" % (T * 4 / 1e9),
            "parallelism": f"replicas{world}"}
IMAD_PER_SM_CLK = 64        # 32-bit integer multiply(-add) results per SM per clock
IMAD_PER_PERMHASH = 4       # two 32x32->64 products (lo and hi halves) per (a*h + b)


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per document of
# the two roofline kernels, from ncu captures (same 11 x 116.8 MB filters as
# the bench).  Reported only while the kernel's sources, comments aside, hash
# to the captured state: a changed kernel reports null.
_CSRC = "paper_2411_04257_gb300/csrc/"
_TRAFFIC = {
    # one launch of 100,000 documents (489.4M tokens): 2,032.8 MB read + 69.8 MB
    # written; the traffic is the tokens read once, so it scales with the
    # documents (tokens) a launch processes
    "k_batched": {"bytes_per_doc": 21026.2,
                  "sources": ["batched_kernels.cuh", "sig_kernels.cuh", "lshb_device.cuh",
                              "bloom_kernels.cuh", "lshb_internal.h", "segment.h"],
                  "sha256": "71ee6a9c8148791df44e1b26758c9865630e0a29b0a90f624769dc36dc83d924",
                  "profile": "profiles/k_batched_pes2o100k_ncu.md"},
    # measured at the bench's launch size, 333,334 documents per launch (the
    # probe's L2 reuse grows with the documents of a launch, so a per-document
    # figure holds for that size): 3,080 MB read + 65 MB written per launch
    "k_probe": {"bytes_per_doc": 9436.8,
                "sources": ["bloom_kernels.cu", "bloom_kernels.cuh", "lshb_device.cuh",
                            "lshb_internal.h"],
                "sha256": "9f4447b299eebe062d0006afd085277cce7a6b0a06dd15fd4488da197d0d261e",
                "profile": "profiles/bloom_kernels_ncu.md"},
}


def _strip_comments(src):
    """C/C++ source without comments and trailing blanks: edits to comments
    leave the fingerprint of a kernel unchanged."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def _sources_sha256(files, read=None):
    h = hashlib.sha256()
    for rel in files:
        if read is None:
            with open(os.path.join(ROOT, _CSRC, rel), encoding="utf-8") as f:
                text = f.read()
        else:
            text = read(rel)
        h.update(_strip_comments(text).encode())
    return h.hexdigest()


def _traffic(kernel, docs_per_launch):
    """Measured DRAM bytes of one launch of `kernel`, or None once it changed."""
    t = _TRAFFIC[kernel]
    if not docs_per_launch or not t["sha256"] or _sources_sha256(t["sources"]) != t["sha256"]:
        return None
    return t["bytes_per_doc"] * docs_per_launch


def _device_peaks(local):
    """Measured issue rates, random-sector rates and the signature stage's own
    ceiling on this GPU (microbench/peaks.cu), or the error that stopped them."""
    try:
        from microbench import peaks
        return peaks.measure(local)
    except Exception as e:  # measurement support, not the product path
        return {"error": repr(e)}


def _sm_max_mhz(clocks):
    """Maximum SM clock: sampled from nvidia-smi during the timed steps, else
    the generated peaks file."""
    if clocks and clocks.get("sm_max_mhz"):
        return float(clocks["sm_max_mhz"])
    peaks, _ = _measured_peaks()
    return float(peaks.get("sm_max_mhz", 2070.0))


def _best_gather(g):
    """(load form, GB/s) of the fastest 4-byte random-sector read form."""
    if not g:
        return None, None
    forms = {k: v for k, v in g.items() if isinstance(v, dict) and "atom" not in k
             and "whole sector" not in k}
    if not forms:
        return None, None
    k = max(forms, key=lambda x: forms[x]["gbs"])
    return k, forms[k]["gbs"]


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


def _probe_roofline(st, dev_peaks, standard_layout=True):
    """The band-major probe kernel k_probe (one launch per chunk, both forms):
    each probe of a band key addresses one 32-byte sector of its band's
    filter; band by band, one 116.8 MB filter at a time, the working set is
    L2-sized.  `peak` is the measured copy bandwidth; the measured random
    4-byte sector reads over a 4 GiB (DRAM) and a 64 MiB (L2) buffer bracket
    what random sectors can attain."""
    if not st or not st["probe_ms"] or not st["probe_sectors"]:
        return None
    peaks, src = _measured_peaks()
    gbs = st["probe_sectors"] * 32 / (st["probe_ms"] / 1e3) / 1e9
    docs_per_launch = st["docs"] / max(1, st["sig_chunks"])
    traffic = _traffic("k_probe", docs_per_launch) if standard_layout else None
    out = {"bound": "hbm", "kernel": "k_probe (band-major)", "achieved": gbs,
           "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
           "traffic": traffic, "algorithmic_bytes_per_launch":
               st["probe_sectors"] * 32 / max(1, st["sig_chunks"]),
           "launch_ms": st["probe_ms"] / max(1, st["sig_chunks"]),
           "peak_source": f"hbm_gbs, {src}",
           "algorithmic_bytes": "32 B per addressed sector: b*k = 187 per document "
                                "(standard layout), b = 11 (blocked layout)"}
    if dev_peaks and "gather_dram" in dev_peaks:
        fd, gd = _best_gather(dev_peaks["gather_dram"])
        fl, gl = _best_gather(dev_peaks["gather_l2"])
        out["random_sector_peaks"] = {"dram_4gib": {"gbs": gd, "load": fd},
                                      "l2_64mib": {"gbs": gl, "load": fl}}
        out["frac_of_random_dram"] = gbs / gd if gd else None
        out["frac_of_random_l2"] = gbs / gl if gl else None
    return out


def _clocks_rejected(c):
    """A timed run that saw a hardware or thermal slowdown, or SM clocks well
    below their maximum with no reason given (a leftover clock lock)."""
    if not c or c.get("sm_mhz") is None:
        return False
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(c.get("reasons", [])):
        return True
    return not c.get("reasons") and c["sm_mhz"] < 0.9 * c["sm_max_mhz"]


def _any_rank(flag, device=None):
    """The flag OR-reduced over ranks, so that all ranks take the same branch."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return bool(flag)
    t = torch.tensor([1.0 if flag else 0.0], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return bool(t.item() > 0)


def _h2d_probe(h_src, d_dst, nbytes=4 << 30):
    """Best of three pinned host->device copies of up to 4 GB, in GB/s."""
    import torch
    n = min(h_src.numel(), d_dst.numel(), nbytes // h_src.element_size())
    if n == 0:
        return None
    st = torch.cuda.current_stream()
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        d_dst[:n].copy_(h_src[:n], non_blocking=True)
        e1.record(st)
        e1.synchronize()
        best = max(best, n * h_src.element_size() / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


def reduce_over_ranks(seconds: float, units: float, device=None):
    """Whole-job timing for N independent replicas (one process per GPU):
    the slowest rank's time and the units every rank processed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return seconds, units
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def _rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _spec(name, rank):
    from synth import corpus
    fac, n, nexp, fp = WORKLOADS[name][:4]
    spec = getattr(corpus, fac)() if fac == "plain_10k" else getattr(corpus, fac)(n_docs=n)
    import dataclasses
    return dataclasses.replace(spec, seed=spec.seed + rank), nexp, fp


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p:
            self.p.terminate()
            self.p.wait()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[0]) for r in rows if len(r) >= 7 and r[0].strip().replace(".", "").isdigit()]
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, n in enumerate(names):
                if len(r) > 3 + i and "Active" in r[3 + i] and "Not" not in r[3 + i]:
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][1]),
                "reasons": sorted(reasons), "samples": len(sm)}


def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return 0
    from oracle import oracle
    from synth import corpus
    spec, nexp, fp = _spec(args.workload, 0)
    t = corpus.build_tables(spec)
    n = args.ref_docs
    off, tok = corpus.generate(spec, 0, n, tables=t)
    times = []
    for i in range(args.warmup + args.steps):
        ix = oracle.OracleIndex(P, BANDS, ROWS, n_expected=nexp, fp_rate=fp, ngram=NGRAM)
        t0 = time.perf_counter()
        ix.dedup(off, tok)
        dt = time.perf_counter() - t0
        ix.close()
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    v = n * len(times) / total
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "docs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": _config(args.workload, world),
            "cpu_baseline": {"value": v, "unit": "docs/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {n} docs of the workload per step "
                                       f"({int(off[-1] - off[0])} tokens)"},
            "e2e": {"value": v, "unit": "docs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _serve_bench(local, seconds_per_load=3.0, n_docs=200_000, seed=0, burst_requests=600):
    """Continuous-batching server over 4 resident indexes (n = 100M each):
    requests of 1-4,096 documents (log-uniform) cut cyclically from a
    serving-shaped corpus (lognormal median 1,000 tokens, 10% near-dups).
    A burst gives the saturation rate; Poisson arrivals at 25/60/90% of it
    give latency percentiles."""
    import dataclasses

    import numpy as np
    import torch

    from paper_2411_04257_gb300 import LSHBloom, LSHBloomServer
    from synth import corpus
    from synth import gpu as sgpu

    spec = dataclasses.replace(corpus.serving_requests(seed=seed), n_docs=n_docs)
    off_d, tok_d = sgpu.DeviceCorpus(spec, torch.device("cuda", local)).generate(0, n_docs)
    torch.cuda.synchronize()
    # the batched form on the same mix, one call over the whole corpus
    # resident in HBM: what the server's saturation compares with
    ixb = LSHBloom(P, BANDS, ROWS, n_expected=100_000_000, fp_rate=1e-5, ngram=NGRAM,
                   device=local)
    for _ in range(3):
        ixb.reset()
        ixb.dedup(off_d, tok_d)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        ixb.reset()
        ixb.dedup(off_d, tok_d)
    torch.cuda.synchronize()
    batched_same_mix = 5 * n_docs / (time.perf_counter() - t0)
    ixb.close()
    off_h = off_d.cpu().numpy().view(np.uint64)
    tok_h = tok_d.cpu().numpy().view(np.uint32)
    del off_d, tok_d
    rnd = np.random.default_rng(seed)
    cursor = [0]

    def next_request():
        D = int(np.exp(rnd.uniform(0.0, np.log(4096.0))))
        D = max(1, min(D, 4096))
        lo = cursor[0] if cursor[0] + D <= n_docs else 0
        cursor[0] = lo + D
        return int(rnd.integers(0, 4)), off_h[lo:lo + D + 1], D

    ixs = [LSHBloom(P, BANDS, ROWS, n_expected=100_000_000, fp_rate=1e-5, ngram=NGRAM,
                    device=local) for _ in range(4)]
    srv = LSHBloomServer(ixs, mem_budget_bytes=4 << 30, max_inflight=64)

    def run(reqs, arrivals):
        t0 = time.perf_counter()
        tickets = []
        for (i, o, D), at in zip(reqs, arrivals):
            while True:
                now = time.perf_counter() - t0
                if now >= at:
                    break
                if at - now > 2e-4:
                    time.sleep((at - now) / 2)
            tickets.append((srv.submit(i, o, tok_h), D))
        lats, docs = [], 0
        for t, D in tickets:
            _, lat = srv.wait(t)
            lats.append(lat)
            docs += D
        span = time.perf_counter() - t0
        return docs / span, np.percentile(lats, 50) / 1e3, np.percentile(lats, 99) / 1e3, len(lats)

    warm = [next_request() for _ in range(64)]
    run(warm, [0.0] * len(warm))
    burst = [next_request() for _ in range(burst_requests)]
    sat, p50, p99, n = run(burst, [0.0] * len(burst))
    out = {"indexes": 4, "n_expected_per_index": 100_000_000, "max_inflight": 64,
           "mem_budget_gb": 4, "saturation_docs_per_s": sat,
           "batched_form_same_mix_docs_per_s": batched_same_mix,
           "burst": {"requests": n, "p50_ms": p50, "p99_ms": p99}, "loads": []}
    mean_docs = 4095.0 / np.log(4096.0)
    for frac in (0.25, 0.60, 0.90):
        rate_req = frac * sat / mean_docs
        n_req = max(50, int(rate_req * seconds_per_load))
        reqs = [next_request() for _ in range(n_req)]
        arrivals = np.cumsum(rnd.exponential(1.0 / rate_req, n_req))
        v, p50, p99, n = run(reqs, arrivals)
        out["loads"].append({"offered_frac": frac, "offered_docs_per_s": frac * sat,
                             "docs_per_s": v, "p50_ms": p50, "p99_ms": p99, "requests": n})
    srv.close()
    for ix in ixs:
        ix.close()
    return out


def _time_steps(fn, steps, warmup, stream, sync, on_start=None):
    import torch
    for _ in range(warmup):
        fn()
    sync()
    if on_start:
        on_start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(steps):
        fn()
    ev[1].record(stream)
    sync()
    return ev[0].elapsed_time(ev[1]) / 1e3


def _timed_mode(ix, off, tok, stream, steps, warmup, sync, local, dev):
    """Timed steps of one index (each step clears the filters and deduplicates
    the batch); a run under a slowdown is measured once more."""
    import torch

    def step():
        ix.reset()
        with torch.cuda.stream(stream):
            ix.dedup_async(off, tok, stream=stream)

    rejected = None
    for attempt in range(2):
        s0 = {}
        with Clocks(local) as ck:
            dt = _time_steps(step, steps, warmup, stream, sync,
                             on_start=lambda: s0.update(ix.stats()))
        clocks = ck.summary()
        s1 = ix.stats()
        if attempt == 0 and _any_rank(_clocks_rejected(clocks), dev):
            rejected = clocks          # measured under a slowdown: once more
            continue
        break
    if rejected is not None:
        clocks["rejected_first_run"] = rejected
    stage = {"sig_ms": s1["sig_ms"] - s0["sig_ms"], "bloom_ms": s1["bloom_ms"] - s0["bloom_ms"],
             "sig_chunks": s1["sig_chunks"] - s0["sig_chunks"],
             "probe_ms": s1["probe_ms"] - s0["probe_ms"],
             "probe_sectors": s1["probe_sectors"] - s0["probe_sectors"],
             "launches": s1["kernel_launches"] - s0["kernel_launches"],
             # reset() at the start of every step clears these two counters:
             # after the last step they hold one step's counts
             "resolve_rounds_per_step": s1["resolve_rounds"],
             "uncertain_docs_per_step": s1["uncertain_docs"]}
    return dt, clocks, stage


def _shingles(off):
    L = off[1:] - off[:-1]
    import torch
    return int(torch.where(L >= NGRAM, L - NGRAM + 1, (L > 0).to(L.dtype)).sum().item())


def _cpu_threaded(off_h, tok_h, nexp, fp, what):
    """The paper's CPU design on the oracle (band keys on all host cores, the
    stream decisions in order on one), on a prefix of the workload."""
    from oracle import oracle
    D = off_h.size - 1
    ix = oracle.OracleIndex(P, BANDS, ROWS, n_expected=nexp, fp_rate=fp, ngram=NGRAM)
    t0 = time.perf_counter()
    flags, used = ix.dedup_threaded(off_h, tok_h, threads=oracle.host_threads())
    dt = time.perf_counter() - t0
    ix.close()
    return {"value": D / dt, "unit": "docs/s", "cores": used,
            "kind": "oracle, threaded: band keys of each 65,536-document block on all "
                    "threads, then the stream decisions in order on one",
            "sample": f"{what}: first {D} docs ({int(off_h[-1] - off_h[0])} tokens), {dt:.1f} s",
            "dups": int(flags.sum())}


def _cpu_oracle(off_h, tok_h, nexp, fp, target_s, what):
    """The oracle as it stands, one thread, on the first documents of
    off_h/tok_h, the count grown until the run takes about target_s/4 .. target_s."""
    from oracle import oracle
    D = off_h.size - 1
    n = min(16, D)
    while True:
        ix = oracle.OracleIndex(P, BANDS, ROWS, n_expected=nexp, fp_rate=fp, ngram=NGRAM)
        t0 = time.perf_counter()
        ix.dedup(off_h[:n + 1], tok_h)
        dt = time.perf_counter() - t0
        ix.close()
        if dt > target_s / 4 or n >= D:
            break
        n = min(D, max(n * 2, int(n * target_s / max(dt, 1e-3) / 2)))
    return {"value": n / dt, "unit": "docs/s", "cores": 1, "kind": "oracle",
            "sample": f"{what}: first {n} docs ({int(off_h[n] - off_h[0])} tokens), {dt:.1f} s"}


def _config_record(name, factory, n_docs, nexp, local, dev, stream, sync, steps, warmup,
                   cpu, threaded_docs, plain=False):
    """One BASELINE configuration on one GPU: its batch resident in HBM, the
    batched form timed over `steps` steps (each clears the filters), and the
    CPU baselines on its first documents."""
    import dataclasses

    import numpy as np

    from paper_2411_04257_gb300 import LSHBloom
    from synth import corpus
    from synth import gpu as sgpu
    spec = dataclasses.replace(getattr(corpus, factory)(), n_docs=n_docs)
    off, tok = sgpu.DeviceCorpus(spec, dev).generate(0, n_docs)
    sync()
    S = _shingles(off)
    rec = {"workload": f"{name}: {n_docs} docs, {int(off[-1].item())} tokens, {S} shingles",
           "n_expected": nexp, "fp_rate": 1e-5, "steps": steps, "warmup": warmup}
    for mode in (["batched", "plain"] if plain else ["batched"]):
        ix = LSHBloom(P, BANDS, ROWS, n_expected=nexp, fp_rate=1e-5, ngram=NGRAM,
                      exec_mode=mode, device=local)
        dt, clocks, st = _timed_mode(ix, off, tok, stream, steps, warmup, sync, local, dev)
        ix.reset()
        flags = ix.dedup_async(off, tok, stream=stream)
        sync()
        r = {"docs_per_s": n_docs * steps / dt, "shingle_hashes_per_s": S * P * steps / dt,
             "ms_per_step": 1e3 * dt / steps,
             "stage_ms_per_step": {"signature": st["sig_ms"] / steps,
                                   "bloom": st["bloom_ms"] / steps,
                                   "probe": st["probe_ms"] / steps},
             "resolve_sweeps_per_step": st["resolve_rounds_per_step"],
             "uncertain_docs_per_step": st["uncertain_docs_per_step"],
             "gpu_launches_per_step": st["launches"] / steps,
             "chunk_docs": ix.stats()["chunk_docs"],
             "dups_per_step": int(flags.sum().item()), "clocks": clocks}
        rec[mode] = r
        ix.close()
    if cpu:
        n = min(n_docs, threaded_docs)
        off_h = off[:n + 1].cpu().numpy().view(np.uint64)
        tok_h = tok[:int(off_h[-1])].cpu().numpy().view(np.uint32)
        del off, tok
        rec["cpu_baseline"] = _cpu_oracle(off_h, tok_h, nexp, 1e-5, 10.0, name)
        rec["cpu_threaded"] = _cpu_threaded(off_h, tok_h, nexp, 1e-5, name)
    return rec


def _billion_record(local, dev, sync, chunk_docs, n_docs, cpu):
    """The billion-document stream in full: documents generated per chunk on
    the device from the counter-based generator (never stored), each chunk
    deduplicated by one call continuing one stream into filters sized for
    n = 1e9 (11 x 3.0 GB).  Throughput counts the dedup calls (CUDA events on
    their stream); the wall time with generation is reported beside it."""
    import numpy as np
    import torch

    from paper_2411_04257_gb300 import LSHBloom
    from synth import corpus
    from synth import gpu as sgpu
    spec = corpus.billion_stream(n_docs=n_docs)
    gen = sgpu.DeviceCorpus(spec, dev)
    ix = LSHBloom(P, BANDS, ROWS, n_expected=1_000_000_000, fp_rate=1e-5, ngram=NGRAM,
                  device=local)
    stream = torch.cuda.Stream(dev)
    dedup_s, docs, shingles, tokens, dups = 0.0, 0, 0, 0, 0
    s0 = ix.stats()
    t0 = time.perf_counter()
    with Clocks(local) as ck:
        for d0 in range(0, n_docs, chunk_docs):
            D = min(chunk_docs, n_docs - d0)
            off, tok = gen.generate(d0, D)
            shingles += _shingles(off)
            tokens += int(tok.numel())
            sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            flags = ix.dedup_async(off, tok, stream=stream)
            e1.record(stream)
            e1.synchronize()
            dedup_s += e0.elapsed_time(e1) / 1e3
            docs += D
            dups += int(flags.sum().item())
            del off, tok, flags
    wall = time.perf_counter() - t0
    s1 = ix.stats()
    ix.close()
    rec = {"workload": f"billion_stream: {docs} docs, {tokens} tokens, {shingles} shingles "
                       f"(generated on the device per chunk of {chunk_docs} docs)",
           "n_expected": 1_000_000_000, "fp_rate": 1e-5, "chunks": (n_docs + chunk_docs - 1)
           // chunk_docs, "docs_per_s": docs / dedup_s, "shingle_hashes_per_s":
               shingles * P / dedup_s, "dedup_s": dedup_s, "wall_s_with_generation": wall,
           "stage_s": {"signature": (s1["sig_ms"] - s0["sig_ms"]) / 1e3,
                       "bloom": (s1["bloom_ms"] - s0["bloom_ms"]) / 1e3},
           "dups": dups, "clocks": ck.summary()}
    if cpu:
        off, tok = gen.generate(0, 1_000_000)
        sync()
        off_h = off.cpu().numpy().view(np.uint64)
        tok_h = tok.cpu().numpy().view(np.uint32)
        del off, tok
        rec["cpu_baseline"] = _cpu_oracle(off_h, tok_h, 1_000_000_000, 1e-5, 10.0,
                                          "billion_stream")
        rec["cpu_threaded"] = _cpu_threaded(off_h, tok_h, 1_000_000_000, 1e-5, "billion_stream")
    return rec


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = _rank_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2411_04257_gb300 import LSHBloom
    from synth import gpu as sgpu

    dev_peaks = None if args.skip_peaks else _device_peaks(local)
    spec, nexp, fp = _spec(args.workload, rank)
    gen = sgpu.DeviceCorpus(spec, dev)
    off, tok = gen.generate(0, spec.n_docs)
    torch.cuda.synchronize()
    D = spec.n_docs
    T = int(off[-1].item())
    shingles = _shingles(off)
    permhashes = shingles * P
    if rank == 0 and (D, T, shingles) != (WORKLOADS[args.workload][1], *WORKLOADS[args.workload][4:]):
        raise RuntimeError(f"generated corpus ({D} docs, {T} tokens, {shingles} shingles) differs "
                           f"from the workload table")
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    stream = torch.cuda.Stream(dev)

    def barrier_sync():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    results = {}
    stage = {}
    modes = ["batched", "plain"] if not args.skip_plain else ["batched"]
    if not args.skip_variants:
        modes += ["batched/blocked", "batched/exact", "batched/weighted"]
    index_bytes = {}
    for mode in modes:
        variant = mode.split("/")[1] if "/" in mode else "standard"
        layout = variant if variant in ("blocked", "exact") else "standard"
        ix = LSHBloom(P, BANDS, ROWS, n_expected=nexp, fp_rate=fp, ngram=NGRAM,
                      exec_mode=mode.split("/")[0], device=local, bloom_layout=layout,
                      band_key="weighted" if variant == "weighted" else "sum")
        st0 = ix.stats()
        index_bytes[layout] = st0["filter_bytes"] * st0["bands"]
        # the layout variants are context: fewer steps
        steps = args.steps if "/" not in mode else min(args.steps, 5)
        warmup = args.warmup if "/" not in mode else min(args.warmup, 2)
        dt, clocks, st = _timed_mode(ix, off, tok, stream, steps, warmup, barrier_sync, local, dev)
        st["docs"] = D * steps
        st["steps"] = steps
        stage[mode] = st
        dt, docs = reduce_over_ranks(dt, float(D * steps), dev)
        _, ph = reduce_over_ranks(dt, float(permhashes * steps), dev)
        ix.reset()
        flags = ix.dedup_async(off, tok, stream=stream)
        torch.cuda.synchronize()
        results[mode] = {"seconds": dt, "steps": steps, "docs_per_s": docs / dt,
                         "shingle_hashes_per_s": ph / dt, "clocks": clocks,
                         "dups_per_step": int(flags.sum().item()),
                         "item_shingles": ix.stats()["item_shingles"]}
        ix.close()

    # --- dominant kernel: the signature stage (persistent kernel), timed with
    # CUDA events on its launching stream inside the timed steps ------------
    sb = stage["batched"]
    sig_s = sb["sig_ms"] / 1e3 / args.steps          # per step
    achieved_imad = IMAD_PER_PERMHASH * permhashes / sig_s
    clocks_b = results["batched"]["clocks"]
    sm_max = _sm_max_mhz(clocks_b)
    peak_imad = sms * IMAD_PER_SM_CLK * sm_max * 1e6
    roofline = {"bound": "alu", "kernel": "k_batched (SHA-1 + MinHash + band keys)",
                "achieved": achieved_imad / 1e12, "peak": peak_imad / 1e12,
                "unit": "T int-mul/s", "frac": achieved_imad / peak_imad,
                "traffic": _traffic("k_batched", D * args.steps / max(1, sb["sig_chunks"])),
                "launch_ms": sb["sig_ms"] / max(1, sb["sig_chunks"]),
                "launches_per_step": sb["sig_chunks"] / args.steps,
                "perm_hashes_per_s": permhashes / sig_s,
                "peak_source": f"{sms} SMs (device) x {IMAD_PER_SM_CLK} IMAD/clk x "
                               f"{sm_max:.0f} MHz (nvidia-smi maximum)"}
    if dev_peaks and "issue" in dev_peaks and dev_peaks["issue"]:
        iss = dev_peaks["issue"]
        roofline["measured_issue_rates"] = {k: v["ops_per_s"] for k, v in iss.items()}
        roofline["frac_of_measured_mad_lo"] = achieved_imad / iss["mad.lo.u32"]["ops_per_s"]
    if dev_peaks and dev_peaks.get("ceiling"):
        both = dev_peaks["ceiling"].get("sha1 + fold")
        fold = dev_peaks["ceiling"].get("fold (P=121, PPL=4)")
        sha = dev_peaks["ceiling"].get("sha1 5-gram windows")
        roofline["ceiling"] = {
            "what": "the same SHA-1 window hash and MinHash fold from registers and shared "
                    "memory, no global memory (microbench/peaks.cu)",
            "sha1_plus_fold_perm_hashes_per_s": both["perm_hashes_per_s"] if both else None,
            "fold_only_perm_hashes_per_s": fold["perm_hashes_per_s"] if fold else None,
            "sha1_only_shingles_per_s": sha["shingles_per_s"] if sha else None,
            "frac": (permhashes / sig_s) / both["perm_hashes_per_s"] if both else None}

    # --- end to end through host buffers --------------------------------------
    e2e = None
    if not args.skip_e2e:
        h_off = torch.empty(D + 1, dtype=torch.int64, pin_memory=True)
        h_tok = torch.empty(T, dtype=torch.int32, pin_memory=True)
        h_off.copy_(off)
        h_tok.copy_(tok)
        h_flags = torch.empty(D, dtype=torch.uint8, pin_memory=True)
        ixe = LSHBloom(P, BANDS, ROWS, n_expected=nexp, fp_rate=fp, ngram=NGRAM,
                       exec_mode="batched", device=local)
        for _ in range(max(1, args.warmup)):
            ixe.reset()
            ixe.dedup(h_off, h_tok, out=h_flags)
        h2d_gbs = _h2d_probe(h_tok, tok)
        rejected = None
        for attempt in range(2):
            barrier_sync()
            s0 = ixe.stats()
            with Clocks(local) as ck:
                t0 = time.perf_counter()
                for _ in range(args.steps):
                    ixe.reset()
                    ixe.dedup(h_off, h_tok, out=h_flags)
                barrier_sync()
                et = time.perf_counter() - t0
            s1 = ixe.stats()
            e2e_clocks = ck.summary()
            if attempt == 0 and _any_rank(_clocks_rejected(e2e_clocks), dev):
                rejected = e2e_clocks
                continue
            break
        if rejected is not None:
            e2e_clocks["rejected_first_run"] = rejected
        et, docs = reduce_over_ranks(et, float(D * args.steps), dev)
        ixe.close()
        e2e = {"value": docs / et, "unit": "docs/s",
               "h2d_bytes_per_step": (D + 1) * 8 + T * 4, "d2h_bytes_per_step": D,
               # context for the number: the pinned-copy bandwidth of this host
               # just before the timed steps, the library's own kernel time of
               # the steps (copies overlap it), and the clocks meanwhile
               "h2d_probe_gbs": h2d_gbs,
               "kernel_ms_per_step": (s1["sig_ms"] + s1["bloom_ms"] - s0["sig_ms"] - s0["bloom_ms"])
                                     / args.steps,
               "chunks_per_step": (s1["sig_chunks"] - s0["sig_chunks"]) / args.steps,
               "h2d_ms_per_step": (s1["h2d_ms"] - s0["h2d_ms"]) / args.steps,
               "h2d_gbs_in_steps": ((s1["h2d_bytes"] - s0["h2d_bytes"])
                                    / max(1e-9, (s1["h2d_ms"] - s0["h2d_ms"]) / 1e3) / 1e9),
               "call_ms_per_step": (s1["call_ms"] - s0["call_ms"]) / args.steps,
               # tokens the kernels read in place from the pinned buffers over
               # the host link (no staging copy), per step
               "host_read_bytes_per_step": (s1["host_read_bytes"] - s0["host_read_bytes"])
                                           / args.steps,
               "clocks": e2e_clocks}
        del h_tok

    # CPU baselines read the first documents of the resident batch
    cpu = cpu_thr = None
    if rank == 0 and not args.skip_cpu:
        n_thr = min(D, args.threaded_docs)
        off_h = off[:n_thr + 1].cpu().numpy().view(np.uint64)
        tok_h = tok[:int(off_h[-1])].cpu().numpy().view(np.uint32)
        cpu = _cpu_oracle(off_h, tok_h, nexp, fp, 12.0, args.workload)
        cpu_thr = _cpu_threaded(off_h, tok_h, nexp, fp, args.workload)
        del off_h, tok_h

    serve = None
    del off, tok
    torch.cuda.empty_cache()
    if not args.skip_serve:
        serve = _serve_bench(local, burst_requests=args.serve_burst)

    # the other configurations: parity cases, measured here as sub-records
    configs = None
    if not args.skip_configs:
        configs = {}
        cpu_cfg = rank == 0 and not args.skip_cpu
        configs["plain_10k"] = _config_record("plain_10k", "plain_10k", 10_000, 10_000, local, dev,
                                              stream, barrier_sync, 50, 5, cpu_cfg, 10_000,
                                              plain=True)
        # 6 warm-up steps: the first five calls of >= 2^22 documents tune the
        # chunk size (one with the largest candidate, then one per candidate)
        configs["pareto_8m"] = _config_record("pareto_8m", "pareto_batched", 8_000_000, 39_000_000,
                                              local, dev, stream, barrier_sync, 5, 6, cpu_cfg,
                                              1_000_000, plain=True)
        torch.cuda.empty_cache()
        configs["billion_stream"] = _billion_record(local, dev, barrier_sync, args.billion_chunk,
                                                    args.billion_docs, cpu_cfg)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    b = results["batched"]
    line = {
        "metric": METRIC,
        "value": b["docs_per_s"], "unit": "docs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * b["seconds"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": _config(args.workload, world),
        "shingle_hashes_per_s": b["shingle_hashes_per_s"],
        "plain": ({"value": results["plain"]["docs_per_s"], "unit": "docs/s",
                   "shingle_hashes_per_s": results["plain"]["shingle_hashes_per_s"]}
                  if "plain" in results else None),
        "dups_per_step": b["dups_per_step"],
        "clocks": b["clocks"],
        "e2e": e2e,
        "gpu_launches": stage["batched"]["launches"],
        "roofline": roofline,
        "stage_ms_per_step": {m: {"signature": v["sig_ms"] / v["steps"],
                                  "bloom": v["bloom_ms"] / v["steps"],
                                  "probe": v["probe_ms"] / v["steps"],
                                  "resolve_sweeps": v["resolve_rounds_per_step"],
                                  "uncertain_docs": v["uncertain_docs_per_step"]}
                              for m, v in stage.items()},
        "roofline_probe": _probe_roofline(stage.get("batched"), dev_peaks),
        "index_variants": ({lay: {"batched_docs_per_s": results[f"batched/{lay}"]["docs_per_s"],
                                  "steps": results[f"batched/{lay}"]["steps"],
                                  "dups_per_step": results[f"batched/{lay}"]["dups_per_step"],
                                  "index_bytes": index_bytes[lay],
                                  "bloom_stage_ms_per_step":
                                      stage[f"batched/{lay}"]["bloom_ms"]
                                      / stage[f"batched/{lay}"]["steps"],
                                  "roofline_probe": _probe_roofline(stage[f"batched/{lay}"],
                                                                    dev_peaks, False)}
                            for lay in ("blocked", "exact")} | {
                               "standard": {"index_bytes": index_bytes["standard"],
                                            "dups_per_step": b["dups_per_step"],
                                            "bloom_stage_ms_per_step":
                                                stage["batched"]["bloom_ms"] / args.steps},
                               # standard filters, weighted band keys (beyond the paper)
                               "weighted_band_keys": {
                                   "batched_docs_per_s": results["batched/weighted"]["docs_per_s"],
                                   "steps": results["batched/weighted"]["steps"],
                                   "dups_per_step": results["batched/weighted"]["dups_per_step"],
                                   "bloom_stage_ms_per_step":
                                       stage["batched/weighted"]["bloom_ms"]
                                       / stage["batched/weighted"]["steps"]}}
                           if not args.skip_variants else None),
        "serve": serve,
        "configs": configs,
        "item_shingles": b["item_shingles"],
        "cpu_baseline": cpu,
        "cpu_threaded": cpu_thr,
        "device_peaks": dev_peaks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pes2o_1m", choices=sorted(WORKLOADS))
    ap.add_argument("--ref-docs", type=int, default=1000)
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--skip-variants", action="store_true",
                    help="skip the blocked filter layout, the exact band-key index and "
                         "weighted band keys")
    ap.add_argument("--skip-configs", action="store_true",
                    help="skip the 10k, 8M Pareto and billion-document configurations")
    ap.add_argument("--skip-peaks", action="store_true", help="skip the peak microbenchmarks")
    ap.add_argument("--threaded-docs", type=int, default=100_000,
                    help="documents of the workload the threaded CPU baseline runs")
    ap.add_argument("--serve-burst", type=int, default=600,
                    help="requests of the serving burst that measures saturation")
    ap.add_argument("--billion-docs", type=int, default=1_000_000_000)
    ap.add_argument("--billion-chunk", type=int, default=4_000_000)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
