#!/usr/bin/env python3
"""Benchmark of the exact GF(p) product, one JSON line on stdout.

Workload: p = 3, m = k = n = 1024, residues i.i.d. uniform in [0, p) (seeded,
synthetic: the paper has no dataset).  One step runs every stage of the hot
path once on that input:

  parameters (host)            gfp_params for every form
  Q-adic dot form, u64 words   gfp_pack(A, rows reversed), gfp_pack(B, columns),
                               gfp_gemm_compressed(dot, u64)
  Q-adic dot form, FP64 words  the same with binary64 words (round-toward-zero)
  right-compressed form, u64   gfp_pack(B, rows), gfp_gemm_compressed(mixed)
                               with REDQ, gfp_unpack(CC)
  classical product            gfp_gemm(plain)
  exact tensor-core forms      gfp_gemm(tc_f16), gfp_gemm(tc_f8), gfp_gemm(tc_mma_s8)

value = (products per step x 2mnk) / step time (every product is the full
C = A B mod p).  Each step is timed alone with CUDA events; a 256 MiB buffer
is written between steps so that no step starts with its inputs in L2.
`forms` gives each form (and each machine word) timed on its own, `batched`
the grouped launch over 4096 adjacency squares, `roofline` the dominant
kernel of the step against its pipe's peak.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gfp|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

P, M, K, N = 3, 1024, 1024, 1024
FLOP = 2.0 * M * N * K
METRIC = "GF(p) GEMM effective 2mnk/s (bit-exact) per form vs plain GPU; % of roofline"
UNIT = "T(2mnk)/s"
WORKLOAD = "Q-adic compressed GEMM and all forms, p=3, m=k=n=1024, uniform residues"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# Throughput ceilings of the pipe each form runs on.  Instruction rates were
# measured on this machine's GB300 by chains of one instruction over 4 CTAs per
# SM (152 SMs at 2.07 GHz); tensor-core rates from MEASURED_PEAKS.json (bf16
# dense burst; fp16 runs at the bf16 rate, e4m3 at twice it).  Each form's
# work is counted in the unit its inner loop issues.
PIPES = {
    "imad": (19.6e12, "IMAD/s (32-bit multiply-add, measured)"),
    "imad_wide": (19.6e12, "IMAD.WIDE/s (32x32->64 multiply-add, measured)"),
    "dp4a": (19.7e12, "dp4a/s (measured)"),
    "mad64": (7.2e12, "64-bit mad.lo/s (measured)"),
    "mad64x2": (3.6e12, "64x64->128 multiply-adds/s (two 64-bit mads each, from the measured mad rate)"),
    "mad64x32": (9.8e12, "64x32-bit multiply-adds/s (two IMADs each, from the measured IMAD rate)"),
    "dfma": (0.625e12, "DFMA/s (nominal FP64 of GB300; a measured chain reached 0.52e12)"),
    "mma_s8": (158e12, "int8 mma.sync ops/s (measured)"),
}


# DRAM bytes of one launch of the dominant kernel (simt_gemm_kernel<DotF64,
# 32, 32, 16, 2, 2> on this step's input), from an ncu capture of this bench:
# 4,212,224 read (CA + CB once) + 0 written (the uint8 C leaves L2 later).
DOTF64_TRAFFIC = 4212224


def form_roofline(ms: float, work: float, pipe: str = None, peak: float = None, unit: str = None):
    """Achieved rate of `work` units in `ms` against a pipe's ceiling."""
    if pipe is not None:
        peak, unit = PIPES[pipe]
    achieved = work / (ms * 1e-3)
    return {"work_per_launch": work, "peak": peak, "unit": unit, "frac": round(achieved / peak, 4)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "gfp_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
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
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the GPU step
# ---------------------------------------------------------------------------
class Step:
    """Every stage of the hot path on one (A, B); buffers allocated once."""

    LAUNCHES = 17   # kernels of this library per step (counted below)

    def __init__(self, gfp, torch, A, B):
        self.gfp, self.torch = gfp, torch
        self.A, self.B = A, B
        dev = A.device
        e = lambda *s, dt=torch.uint8: torch.empty(*s, dtype=dt, device=dev)
        self.d64, self.Q64, _ = gfp.gfp_params(P, M, K, N, "dot", "u64")
        self.df, self.Qf, _ = gfp.gfp_params(P, M, K, N, "dot", "f64")
        self.dm, self.Qm, _ = gfp.gfp_params(P, M, K, N, "mixed", "u64")
        kc64 = -(-K // (self.d64 + 1))
        kcf = -(-K // (self.df + 1))
        self.CA64 = e((M, kc64), dt=torch.int64)
        self.CB64 = e((kc64, N), dt=torch.int64)
        self.CAf = e((M, kcf), dt=torch.float64)
        self.CBf = e((kcf, N), dt=torch.float64)
        ncm = -(-N // (self.dm + 1))
        self.CBr = e((K, ncm), dt=torch.int64)
        self.CC = e((M, ncm), dt=torch.int64)
        self.outs = {name: e((M, N)) for name in ("dot_u64", "dot_f64", "mixed_u64", "plain", "tc_f16",
                                                  "tc_f8", "tc_mma_s8")}
        self.ws16 = e(gfp.gfp_gemm_workspace_size(P, M, K, N, "tc_f16"))
        self.wsf8 = e(gfp.gfp_gemm_workspace_size(P, M, K, N, "tc_f8"))
        self.ws8 = e(gfp.gfp_gemm_workspace_size(P, M, K, N, "tc_mma_s8"))
        self.dom = None   # (start, end) events around the dominant kernel

    def run(self, dom_events=None, done=None):
        """One step.  `done(name)`, if given, is called as soon as the launch
        that completes output `name` has been issued (to start its copy)."""
        g = self.gfp
        done = done or (lambda name: None)
        # parameters (host)
        d64, Q64, _ = g.gfp_params(P, M, K, N, "dot", "u64")
        df, Qf, _ = g.gfp_params(P, M, K, N, "dot", "f64")
        dm, Qm, _ = g.gfp_params(P, M, K, N, "mixed", "u64")
        # dot form, u64 words: 3 launches
        g.gfp_pack(P, self.A, d64, Q64, "rows_rev", "u64", out=self.CA64)
        g.gfp_pack(P, self.B, d64, Q64, "cols", "u64", out=self.CB64)
        g.gfp_gemm_compressed(P, M, K, N, d64, Q64, "dot", "u64", self.CA64, self.CB64, out=self.outs["dot_u64"])
        done("dot_u64")
        # dot form, FP64 words: 3 launches (the product is the step's dominant kernel)
        g.gfp_pack(P, self.A, df, Qf, "rows_rev", "f64", out=self.CAf)
        g.gfp_pack(P, self.B, df, Qf, "cols", "f64", out=self.CBf)
        if dom_events is not None:
            dom_events[0].record()
        g.gfp_gemm_compressed(P, M, K, N, df, Qf, "dot", "f64", self.CAf, self.CBf, out=self.outs["dot_f64"])
        if dom_events is not None:
            dom_events[1].record()
        done("dot_f64")
        # right-compressed form with REDQ: 3 launches
        g.gfp_pack(P, self.B, dm, Qm, "rows", "u64", out=self.CBr)
        g.gfp_gemm_compressed(P, M, K, N, dm, Qm, "mixed", "u64", self.A, self.CBr, out=self.CC)
        g.gfp_unpack(P, self.CC, M, N, dm, Qm, "rows", "u64", out=self.outs["mixed_u64"])
        done("mixed_u64")
        # classical product: 1 launch
        g.gfp_gemm(P, self.A, self.B, "plain", out=self.outs["plain"])
        done("plain")
        # tensor-core forms: 3 + 2 + 3 launches (operand conversion, product; the
        # fp8 form converts only B for p < 16)
        g.gfp_gemm(P, self.A, self.B, "tc_f16", out=self.outs["tc_f16"], workspace=self.ws16)
        done("tc_f16")
        g.gfp_gemm(P, self.A, self.B, "tc_f8", out=self.outs["tc_f8"], workspace=self.wsf8)
        done("tc_f8")
        g.gfp_gemm(P, self.A, self.B, "tc_mma_s8", out=self.outs["tc_mma_s8"], workspace=self.ws8)
        done("tc_mma_s8")

    @property
    def products(self):
        return len(self.outs)


def event_time(torch, fn, reps, flush):
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def forms_breakdown(gfp, torch, A, B, flush, plain_ms):
    """Each form and word timed on its own (median of 7, L2 flushed), with
    its fraction of the ceiling of the pipe it runs on."""
    out = {}
    dev = A.device
    bf16 = (measured_peaks().get("bf16_tflops") or 1900.0) * 1e12
    hbm = (measured_peaks().get("hbm_gbs") or 6800.0) * 1e9

    def rec(name, ms, roof=None, **extra):
        r = {"ms": round(ms, 5), "value": round(FLOP / ms / 1e9, 3), "speedup_vs_plain": round(plain_ms / ms, 3)}
        r.update(extra)
        if roof is not None:
            r["roofline"] = roof
        out[name] = r

    tc_roof = {"plain": lambda ms: form_roofline(ms, M * N * K, "imad"),
               "dp4a": lambda ms: form_roofline(ms, M * N * -(-K // 4), "dp4a"),
               "tc_mma_s8": lambda ms: form_roofline(ms, FLOP, "mma_s8"),
               "tc_f16": lambda ms: form_roofline(ms, FLOP, peak=bf16, unit="fp16 tcgen05 flops/s (bf16 dense, measured)"),
               "tc_f8": lambda ms: form_roofline(ms, FLOP, peak=2 * bf16,
                                                 unit="e4m3 tcgen05 flops/s (2 x measured bf16 dense)")}
    for algo in ("plain", "dp4a", "tc_mma_s8", "tc_f16", "tc_f8"):
        ws = torch.empty(max(1, gfp.gfp_gemm_workspace_size(P, M, K, N, algo)), dtype=torch.uint8, device=dev)
        C = torch.empty((M, N), dtype=torch.uint8, device=dev)
        ms = event_time(torch, lambda: gfp.gfp_gemm(P, A, B, algo, out=C, workspace=ws), 7, flush)
        rec(algo, ms, tc_roof[algo](ms))
    word_pipe = {"u64": "mad64", "u64x128": "mad64x2", "u32w": "imad_wide", "u32": "imad", "f64": "dfma"}
    for word, kb in (("u64", 0), ("u64x128", 0), ("u32w", 0), ("u32", 0), ("f64", 0), ("u32", 60),
                     ("u32w", 140)):
        d, Q, kbr = gfp.gfp_params(P, M, K, N, "dot", word, kb=kb)
        CA = gfp.gfp_pack(P, A, d, Q, "rows_rev", word)
        CB = gfp.gfp_pack(P, B, d, Q, "cols", word)
        C = torch.empty((M, N), dtype=torch.uint8, device=dev)
        t_mm = event_time(torch, lambda: gfp.gfp_gemm_compressed(P, M, K, N, d, Q, "dot", word, CA, CB, out=C, kb=kbr), 7, flush)

        def full():
            gfp.gfp_pack(P, A, d, Q, "rows_rev", word, out=CA)
            gfp.gfp_pack(P, B, d, Q, "cols", word, out=CB)
            gfp.gfp_gemm_compressed(P, M, K, N, d, Q, "dot", word, CA, CB, out=C, kb=kbr)
        t_full = event_time(torch, full, 7, flush)
        name = "dot_%s" % word + ("_kb%d" % kbr if kbr else "")
        rec(name, t_mm, form_roofline(t_mm, M * N * -(-K // (d + 1)), word_pipe[word]),
            d_plus_1=d + 1, t=Q.bit_length() - 1, kb=kbr,
            with_packing_ms=round(t_full, 5), with_packing_value=round(FLOP / t_full / 1e9, 3))
    # the autotuner's pick of (word, d, Q, k-block) for this shape (untimed search)
    best, cands = gfp.gfp_dot_autotune(P, M, K, N)
    word, d, Q, kbr = best["word"], best["d"], best["Q"], best["kb"]
    CA = gfp.gfp_pack(P, A, d, Q, "rows_rev", word)
    CB = gfp.gfp_pack(P, B, d, Q, "cols", word)
    C = torch.empty((M, N), dtype=torch.uint8, device=dev)
    ms = event_time(torch, lambda: gfp.gfp_gemm_compressed(P, M, K, N, d, Q, "dot", word, CA, CB, out=C, kb=kbr), 7, flush)
    rec("dot_autotuned", ms, form_roofline(ms, M * N * -(-K // (d + 1)), word_pipe[word]), word=word,
        d_plus_1=d + 1, t=Q.bit_length() - 1, kb=kbr, candidates=len(cands))
    for word in ("u64", "f64"):
        d, Q, _ = gfp.gfp_params(P, M, K, N, "mixed", word)
        CB = gfp.gfp_pack(P, B, d, Q, "rows", word)
        CC = torch.empty((M, -(-N // (d + 1))), dtype=gfp.WORD_DTYPE[word], device=dev)
        ms = event_time(torch, lambda: gfp.gfp_gemm_compressed(P, M, K, N, d, Q, "mixed", word, A, CB, out=CC), 7, flush)
        rec("mixed_%s" % word, ms, form_roofline(ms, M * K * -(-N // (d + 1)), "mad64x32" if word == "u64" else "dfma"),
            d_plus_1=d + 1, t=Q.bit_length() - 1)
    # left (Table 2) and full (Section 4) compression, u64 words, product only
    d, Q, _ = gfp.gfp_params(P, M, K, N, "left", "u64")
    CA = gfp.gfp_pack(P, A, d, Q, "cols", "u64")
    CC = torch.empty((-(-M // (d + 1)), N), dtype=torch.int64, device=dev)
    ms = event_time(torch, lambda: gfp.gfp_gemm_compressed(P, M, K, N, d, Q, "left", "u64", CA, B, out=CC), 7, flush)
    rec("left_u64", ms, form_roofline(ms, -(-M // (d + 1)) * K * N, "mad64x32"), d_plus_1=d + 1, t=Q.bit_length() - 1)
    dq, dth, Q = gfp.gfp_params_full(P, M, K, N, "u64")
    CA = gfp.gfp_pack(P, A, dq, Q, "cols", "u64")
    CB = gfp.gfp_pack(P, B, dth, Q ** (dq + 1), "rows", "u64")
    CC = torch.empty((-(-M // (dq + 1)), -(-N // (dth + 1))), dtype=torch.int64, device=dev)
    ms = event_time(torch, lambda: gfp.gfp_gemm_full(P, M, K, N, dq, dth, Q, "u64", CA, CB, out=CC), 7, flush)
    rec("full_u64", ms, form_roofline(ms, -(-M // (dq + 1)) * K * -(-N // (dth + 1)), "mad64"),
        dq=dq, dth=dth, t=Q.bit_length() - 1)
    # conversions: pack A reversed into u64 words, bytes moved per launch
    d, Q, _ = gfp.gfp_params(P, M, K, N, "dot", "u64")
    CA = gfp.gfp_pack(P, A, d, Q, "rows_rev", "u64")
    t = event_time(torch, lambda: gfp.gfp_pack(P, A, d, Q, "rows_rev", "u64", out=CA), 7, flush)
    byts = M * K + CA.numel() * 8
    out["pack_rows_rev_u64"] = {"ms": round(t, 5), "GB_per_s": round(byts / t / 1e6, 1), "bytes": byts,
                                "roofline": form_roofline(t, byts, peak=hbm, unit="bytes/s (measured HBM copy)")}
    return out


def batched_measure(gfp, torch, flush):
    """4096 squares of adjacency matrices in one grouped launch (CUDA graph)."""
    from paper_0803_1975_gb300 import inputs
    probs = inputs.batched_problems()
    dev = torch.device("cuda")
    items = []
    flops = 0.0
    for p, A in probs:
        Ad = torch.from_numpy(A).to(dev)
        n = A.shape[0]
        items.append((p, Ad, Ad, torch.empty((n, n), dtype=torch.uint8, device=dev)))
        flops += 2.0 * n ** 3
    arr, cnt = gfp.make_problems(items)
    need = gfp.gfp_batched_workspace_size(arr, cnt)
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    table = gfp.gfp_batched_autotune(arr, cnt, workspace=ws)    # untimed: tile kind per size bucket
    gfp.gfp_batched_prepare(arr, cnt, "auto", ws)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        gfp.gfp_batched_launch(ws)      # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        gfp.gfp_batched_launch(ws)
    ms = event_time(torch, graph.replay, 7, flush)
    # kinds in use: the tuned kind of every size bucket that holds a problem
    kinds = set()
    for p, A in probs:
        n = A.shape[0]
        b = 0 if n <= 32 else 1 if n <= 64 else 2 if n <= 128 else 3 if n <= 256 else 4 if n <= 512 else 5
        k = table[b]
        kinds.add(k if k >= 0 else (4 if p < 16 else 0))
    kernels = 1 + (1 if kinds & {0, 1, 2, 3} else 0) + (1 if 4 in kinds else 0)
    return {"problems": cnt, "sum_2n3": flops, "ms": round(ms, 4), "value": round(flops / ms / 1e9, 3),
            "unit": UNIT, "kernels_per_replay": kernels,
            "autotuned_kinds": [gfp.BATCHED_KINDS.get(v, None) for v in table],
            "note": "one graph replay = operand conversion kernel, then one persistent grouped kernel per "
                    "engine in use: tcgen05 e4m3 tiles (p < 16) and/or mma.sync / Q-adic SIMT tiles"}


# ---------------------------------------------------------------------------
def cpu_oracle_rate(A, B, budget_s=10.0):
    """The oracle (plain C triple loop over all host cores) on the same
    product; repeated until about budget_s of CPU time."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    t0 = time.time()
    oracle.gemm(P, A, B, threads=cores)
    one = time.time() - t0
    reps = max(1, int(budget_s / max(one, 1e-3)) - 1)
    reps = min(reps, 50)
    t0 = time.time()
    for _ in range(reps):
        oracle.gemm(P, A, B, threads=cores)
    per = (time.time() - t0) / reps
    return FLOP / per / 1e12, cores, "%d full %dx%dx%d products (p=%d) after one untimed" % (reps, M, K, N, P), per


def run_reference(args, rank, world):
    """--impl reference: the oracle as it stands, timed on the host cores."""
    if rank != 0:
        return
    from paper_0803_1975_gb300 import inputs
    import oracle
    oracle.build()
    g = inputs.rng(2, 0)
    A = inputs.residues(g, P, M, K)
    B = inputs.residues(g, P, K, N)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.gemm(P, A, B, threads=cores)
    ts = []
    for _ in range(args.steps):
        t0 = time.time()
        oracle.gemm(P, A, B, threads=cores)
        ts.append(time.time() - t0)
    per = float(np.sum(ts)) / args.steps
    v = FLOP / per / 1e12
    line = {"metric": METRIC, "value": round(v, 4), "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "p": P, "m": M, "k": K, "n": N},
            "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one full %dx%dx%d product per step" % (M, K, N)},
            "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gfp", choices=["gfp", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the per-form and batched breakdowns")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_0803_1975_gb300 import build as gbuild
    from paper_0803_1975_gb300 import gfp, inputs
    from paper_0803_1975_gb300.dist import max_over_ranks

    gbuild.build()
    gfp.load()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # every rank runs its own replica of the workload (independent products)
    g = inputs.rng(2, 0)
    A_h = inputs.residues(g, P, M, K)
    B_h = inputs.residues(g, P, K, N)
    A = torch.from_numpy(A_h).cuda()
    B = torch.from_numpy(B_h).cuda()
    step = Step(gfp, torch, A, B)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        step.run()
    torch.cuda.synchronize()

    # correctness of the step's outputs (cheap check against one oracle product on rank 0)
    import oracle
    oracle.build()
    ref = oracle.gemm(P, A_h, B_h, threads=os.cpu_count() or 1)
    for name, C in step.outs.items():
        if not (C.cpu().numpy() == ref).all():
            raise SystemExit("bench: %s result differs from the oracle" % name)

    clocks = Clocks(local)
    clocks.start()
    barrier()
    step_ms, dom_ms = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step.run(dom_events=(d0, d1))
        e1.record()
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        dom_ms.append(d0.elapsed_time(d1))
    barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(float(np.sum(step_ms)), device="cuda")
    ms_per_step = total_ms / args.steps
    value = world * step.products * FLOP / ms_per_step / 1e9

    # end to end: pinned host inputs -> device -> all forms -> results to pinned host memory;
    # each result is copied on a second stream as soon as its product is done
    # (ordered by an event), overlapping the copies with the later products
    A_pin = torch.from_numpy(A_h).pin_memory()
    B_pin = torch.from_numpy(B_h).pin_memory()
    outs_pin = {k: torch.empty((M, N), dtype=torch.uint8).pin_memory() for k in step.outs}
    copy_stream = torch.cuda.Stream()

    def copy_out(name):
        ev = torch.cuda.Event()
        ev.record()
        copy_stream.wait_event(ev)
        with torch.cuda.stream(copy_stream):
            outs_pin[name].copy_(step.outs[name], non_blocking=True)

    barrier()
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        A.copy_(A_pin, non_blocking=True)
        B.copy_(B_pin, non_blocking=True)
        step.run(done=copy_out)
        torch.cuda.current_stream().wait_stream(copy_stream)
        e1.record()
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    barrier()
    e2e_per = max_over_ranks(float(np.mean(e2e_ms)), device="cuda")
    for k_, C in outs_pin.items():
        if not (C.numpy() == ref).all():
            raise SystemExit("bench: end-to-end %s result differs from the oracle" % k_)

    # roofline of the dominant kernel: the FP64 dot product (DFMA pipe)
    kcf = -(-K // (step.df + 1))
    dfma = M * N * kcf
    dom_avg = float(np.mean(dom_ms))
    achieved = 2.0 * dfma / dom_avg / 1e9            # TFLOP/s (FP64, 2 per fused multiply-add)
    fp64_peak = 1.25                                   # nominal FP64 of GB300 (TFLOP/s)
    roofline = {"kernel": "simt_gemm_kernel<DotF64> (dot form, FP64 words)", "bound": "alu",
                "achieved": round(achieved, 4), "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": round(achieved / fp64_peak, 4), "peak_source": "nominal FP64 rate of GB300 (no measured FP64 peak in MEASURED_PEAKS.json)",
                "traffic": DOTF64_TRAFFIC, "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of "
                "one launch of this kernel in this step; algorithmic operand bytes %d" % (8 * kcf * (M + N)), "launch_ms": round(dom_avg, 5),
                "algorithmic_flops_per_launch": 2 * dfma,
                "share_of_step": round(dom_avg / (float(np.mean(step_ms))), 3)}

    extras = {}
    if rank == 0 and not args.no_extras:
        plain_ms = event_time(torch, lambda: gfp.gfp_gemm(P, A, B, "plain", out=step.outs["plain"]), 7, flush)
        extras["forms"] = forms_breakdown(gfp, torch, A, B, flush, plain_ms)
        try:
            extras["batched"] = batched_measure(gfp, torch, flush)
        except gfp.GfpError as e:
            extras["batched"] = {"unavailable": str(e)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample, _ = cpu_oracle_rate(A_h, B_h)
        cpu = {"value": round(v, 5), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        peaks = measured_peaks()
        line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/u32/u64/f64/f16",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "p": P, "m": M, "k": K, "n": N,
                           "products_per_step": step.products,
                           "l2": "256 MiB buffer written between timed steps (flush)",
                           "replicas": world},
                "e2e": {"value": round(world * step.products * FLOP / e2e_per / 1e9, 3), "unit": UNIT,
                        "ms_per_step": round(e2e_per, 5),
                        "h2d_bytes_per_step": 2 * M * K, "d2h_bytes_per_step": step.products * M * N},
                "gpu_launches": Step.LAUNCHES * args.steps,
                "roofline": roofline,
                "clocks": clk,
                "cpu_baseline": cpu,
                "measured_peaks": {"hbm_gbs": peaks.get("hbm_gbs"), "bf16_tflops": peaks.get("bf16_tflops")}}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
