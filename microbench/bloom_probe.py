"""Driver for ncu captures of the Bloom-stage kernels (k_probe, k_insert).

Generates the heavy-tailed Pareto-shaped batch (synth.corpus.pareto_batched)
on the device, then deduplicates it with LSHBloom(121, 11, 11, n = 39M,
p = 1e-5) in launches of --chunk-docs documents: 11 filters of 116.8 MB,
larger than L2 together, one band's filter about L2's size, as in the
benchmark.  Short documents keep the device footprint to a few GB, so a
multi-pass capture of one launch stays small.

    python -m microbench.bloom_probe --chunk-docs 333334 [--docs 8000000]
        [--layout standard|blocked|exact] [--repeat 1]

Prints one JSON line (documents, launches, duplicates, per-call wall times, stage
times).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--docs", type=int, default=8_000_000)
    ap.add_argument("--chunk-docs", type=int, default=1 << 20)
    ap.add_argument("--layout", default="standard", choices=["standard", "blocked", "exact"])
    ap.add_argument("--repeat", type=int, default=1)
    args = ap.parse_args(argv)

    import torch

    from paper_2411_04257_gb300 import LSHBloom
    from synth import corpus
    from synth import gpu as sgpu
    dev = torch.device("cuda:0")
    spec = dataclasses.replace(corpus.pareto_batched(), n_docs=args.docs)
    off, tok = sgpu.DeviceCorpus(spec, dev).generate(0, args.docs)
    torch.cuda.synchronize()
    ix = LSHBloom(121, 11, 11, n_expected=39_000_000, fp_rate=1e-5, ngram=5,
                  max_batch_docs=args.chunk_docs, bloom_layout=args.layout, device=0)
    dups, call_ms = [], []
    for _ in range(args.repeat):
        ix.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        flags = ix.dedup(off, tok)
        call_ms.append(1e3 * (time.perf_counter() - t0))
        dups.append(int(flags.sum().item()))
    st = ix.stats()
    ix.close()
    print(json.dumps({"docs": args.docs, "tokens": int(off[-1].item()),
                      "chunk_docs": st["chunk_docs"], "layout": args.layout,
                      "repeat": args.repeat, "dups": dups, "call_ms": call_ms,
                      "pipelined_chunks": st["pipelined_chunks"],
                      "launches": st["kernel_launches"], "sig_ms": st["sig_ms"],
                      "bloom_ms": st["bloom_ms"], "probe_ms": st["probe_ms"]}))


if __name__ == "__main__":
    main()
