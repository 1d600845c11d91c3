"""Run one form of C = A B mod p on seeded uniform residues and report its
time (CUDA events, L2 flushed between repetitions) and effective 2mnk/s.

    python -m paper_0803_1975_gb300.run_case --form tc_f16 --p 3 --size 8192 --reps 3
    python -m paper_0803_1975_gb300.run_case --form dot --word u32 --kb 60 --size 1024

Forms: plain, dp4a, tc_mma_s8, tc_f16, tc_f8, tc_e2m1 (gfp_gemm); dot, mixed, left
(gfp_gemm_compressed, after packing); full (gfp_gemm_full, 64-bit words); winograd (the 64-bit dot form with
--levels of Strassen-Winograd on the words); batched (the 4096-problem adjacency
workload, one prepared launch); pack_rows_rev, pack_cols, pack_rows,
unpack_rows (the conversions of A, reported in GB/s of bytes moved).  Useful
for profiling one kernel.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import gfp, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--form", default="tc_f16")
    ap.add_argument("--word", default="u64")
    ap.add_argument("--kb", type=int, default=0)
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--size", type=int, default=1024)
    ap.add_argument("--m", type=int, default=0)
    ap.add_argument("--k", type=int, default=0)
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--algo", default="auto", help="batched: auto, tc_f16, tc_f8 or dot32")
    ap.add_argument("--levels", type=int, default=1, help="winograd: Strassen-Winograd levels")
    ap.add_argument("--primes", default="", help="batched: comma-separated primes replacing the workload's "
                                                 "p in {3, 5, 7} (cycled; 0/1 matrices are residues for any p)")
    ap.add_argument("--symmetric", action="store_true",
                    help="batched: declare B = A^T (true for the adjacency squares), one staged copy of A")
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--graph", type=int, default=0,
                    help="capture this many calls in one CUDA graph and report the time per call of its "
                         "replay (launch overhead removed; the operands stay in L2 between the calls)")
    a = ap.parse_args()
    m = a.m or a.size
    k = a.k or a.size
    n = a.n or a.size
    p = a.p
    g = inputs.rng(3, p)
    A = torch.from_numpy(inputs.residues(g, p, m, k)).cuda()
    B = torch.from_numpy(inputs.residues(g, p, k, n)).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    if a.form in ("plain", "dp4a", "tc_mma_s8", "tc_f16", "tc_f8", "tc_e2m1"):
        ws = torch.empty(max(1, gfp.gfp_gemm_workspace_size(p, m, k, n, a.form)), dtype=torch.uint8,
                         device="cuda")
        C = torch.empty((m, n), dtype=torch.uint8, device="cuda")
        fn = lambda: gfp.gfp_gemm(p, A, B, a.form, out=C, workspace=ws)
    elif a.form == "dot":
        d, Q, kb = gfp.gfp_params(p, m, k, n, "dot", a.word, kb=a.kb)
        CA = gfp.gfp_pack(p, A, d, Q, "rows_rev", a.word)
        CB = gfp.gfp_pack(p, B, d, Q, "cols", a.word)
        C = torch.empty((m, n), dtype=torch.uint8, device="cuda")
        fn = lambda: gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "dot", a.word, CA, CB, out=C, kb=kb)
    elif a.form in ("pack_rows_rev", "pack_cols", "pack_rows", "unpack_rows"):
        d, Q, _ = gfp.gfp_params(p, m, k, n, "dot", a.word)
        lay = a.form.split("_", 1)[1]
        if a.form == "unpack_rows":
            W = gfp.gfp_pack(p, A, d, Q, "rows", a.word)
            X = torch.empty((m, k), dtype=torch.uint8, device="cuda")
            fn = lambda: gfp.gfp_unpack(p, W, m, k, d, Q, "rows", a.word, out=X)
        else:
            W = gfp.gfp_pack(p, A, d, Q, lay, a.word)
            fn = lambda: gfp.gfp_pack(p, A, d, Q, lay, a.word, out=W)
        pack_bytes = m * k + W.numel() * W.element_size()
    elif a.form == "batched":
        # the 4096-problem adjacency workload, one prepared schedule replayed
        items = []
        primes = [int(x) for x in a.primes.split(",") if x]
        for i, (pp, Ah) in enumerate(inputs.batched_problems()):
            if primes:
                pp = primes[i % len(primes)]
            Ad = torch.from_numpy(Ah).cuda()
            items.append((pp, Ad, Ad, torch.empty(Ah.shape, dtype=torch.uint8, device="cuda")))
        arr, cnt = gfp.make_problems(items, flags=gfp.PROBLEM_B_IS_A_T if a.symmetric else 0)
        ws = torch.empty(gfp.gfp_batched_workspace_size(arr, cnt), dtype=torch.uint8, device="cuda")
        gfp.gfp_batched_prepare(arr, cnt, a.algo, ws)
        m = k = n = 0
        flops_total = sum(2.0 * it[1].shape[0] ** 3 for it in items)
        fn = lambda: gfp.gfp_batched_launch(ws)
    elif a.form == "winograd":
        # the dot form in 64-bit words with Strassen-Winograd levels on the words
        d, Q, _ = gfp.gfp_params(p, m, k, n, "dot", "u64")
        CA = gfp.gfp_pack(p, A, d, Q, "rows_rev", "u64")
        CB = gfp.gfp_pack(p, B, d, Q, "cols", "u64")
        C = torch.empty((m, n), dtype=torch.uint8, device="cuda")
        ws = torch.empty(gfp.gfp_winograd_workspace_size(m, k, n, d, a.levels), dtype=torch.uint8, device="cuda")
        fn = lambda: gfp.gfp_gemm_compressed_winograd(p, m, k, n, d, Q, CA, CB, levels=a.levels, out=C,
                                                      workspace=ws)
    elif a.form == "mixed":
        d, Q, _ = gfp.gfp_params(p, m, k, n, "mixed", a.word)
        CB = gfp.gfp_pack(p, B, d, Q, "rows", a.word)
        C = torch.empty((m, -(-n // (d + 1))), dtype=gfp.WORD_DTYPE[a.word], device="cuda")
        fn = lambda: gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "mixed", a.word, A, CB, out=C)
    elif a.form == "left":
        # left compression (Table 2): A packed along m (column words) times uncompressed B
        d, Q, _ = gfp.gfp_params(p, m, k, n, "left", "u64")
        CA = gfp.gfp_pack(p, A, d, Q, "cols", "u64")
        C = torch.empty((-(-m // (d + 1)), n), dtype=torch.int64, device="cuda")
        fn = lambda: gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "left", "u64", CA, B, out=C)
    elif a.form == "full":
        # full compression (Section 4): A along m in base Q, B along n in base Q^(dq+1)
        dq, dth, Q = gfp.gfp_params_full(p, m, k, n, "u64")
        CA = gfp.gfp_pack(p, A, dq, Q, "cols", "u64")
        CB = gfp.gfp_pack(p, B, dth, Q ** (dq + 1), "rows", "u64")
        C = torch.empty((-(-m // (dq + 1)), -(-n // (dth + 1))), dtype=torch.int64, device="cuda")
        fn = lambda: gfp.gfp_gemm_full(p, m, k, n, dq, dth, Q, "u64", CA, CB, out=C)
    else:
        raise SystemExit("unknown form %s" % a.form)
    for _ in range(a.warmup):
        fn()
    calls = 1
    if a.graph > 0:
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(a.graph):
                fn()
        calls = a.graph
        fn = graph.replay
        fn()
    ts = []
    for _ in range(a.reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.median(ts)) / calls
    if a.form.startswith(("pack", "unpack")):
        print(json.dumps({"form": a.form, "word": a.word, "p": p, "rows": m, "cols": k, "ms": round(ms, 5),
                          "bytes": pack_bytes, "GB_per_s": round(pack_bytes / ms / 1e6, 1)}))
        return
    flops = flops_total if a.form == "batched" else 2.0 * m * n * k
    print(json.dumps({"form": a.form, "word": a.word, "algo": a.algo, "levels": a.levels, "p": p, "m": m, "k": k, "n": n, "ms": round(ms, 5),
                      "T_2mnk_per_s": round(flops / ms / 1e9, 3), "graph_calls": a.graph}))


if __name__ == "__main__":
    main()
