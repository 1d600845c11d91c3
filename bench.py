#!/usr/bin/env python3
"""Benchmark of the exact GF(p) product, one JSON line on stdout.

Workload (the headline): every form of C = A B mod p at p = 5,
m = k = n = 16384, residues i.i.d. uniform in [0, p) (seeded, synthetic: the
paper has no dataset).  One step runs each form once on that input:

  classical product            gfp_gemm(plain): one 32-bit multiply-add per term
  classical product on dp4a    gfp_gemm(dp4a): four byte products per instruction
  Q-adic dot form, u64 words   gfp_pack(A, rows reversed), gfp_pack(B, columns),
                               gfp_gemm_compressed(dot, u64)
  Q-adic dot form, tuned       the same with the word, d, Q and k-block the
                               dot-form autotuner picks for this shape
  right-compressed form, u64   gfp_pack(B, rows), gfp_gemm_compressed(mixed)
                               with REDQ, gfp_unpack(CC)
  exact tensor-core forms      gfp_gemm(tc_mma_s8), gfp_gemm(tc_f16),
                               gfp_gemm(tc_f8), gfp_gemm(tc_e2m1)

value = (products per step x 2mnk) / step time (every product is the full
C = A B mod p, checked bit for bit before timing).  Each step is timed with
CUDA events on the launching stream; the operands (256 MiB each) are larger
than L2 and a 256 MiB buffer is also written between steps.  `forms` gives
each form's time inside the step, its rate, its speedup over both classical
products and its kernel's fraction of the pipe it runs on; `roofline` is the
step's dominant kernel.  Extra keys carry the other workloads:
`compressed_1024` (p = 3, 1024^3, every machine word including FP64),
`tensor_core_8192` (p in {3, 31, 251}, 8192^3), `reduce_compress` (the dot
product with ReduceAndCompress fused, against a separate packing),
`pack_unpack` (the conversions against HBM) and
`batched` (4096 adjacency squares in one graph replay).

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

P, M, K, N = 5, 16384, 16384, 16384
FLOP = 2.0 * M * N * K
METRIC = "GF(p) GEMM effective 2mnk/s (bit-exact) per form vs plain GPU; % of roofline"
UNIT = "T(2mnk)/s"
WORKLOAD = "all forms, p=5, m=k=n=16384, residues i.i.d. uniform in [0,p)"
SEED = (5, 0)                 # inputs.rng(workload 5, trial 0)
ORACLE_ROWS = 16              # rows of the product the reference arm's oracle computes per step


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def config_dict():
    """The workload description shared by both arms of the benchmark."""
    return {"workload": WORKLOAD, "p": P, "m": M, "k": K, "n": N,
            "l2": "operands of 256 MiB each (larger than L2) and a 256 MiB buffer written between steps"}


# Throughput ceilings of the pipes the CUDA-core forms run on, measured on
# this GPU by the library's instruction-rate probe (gfp_pipe_rates: chains of
# one instruction, 32 warps per SM).  Each form's work is counted in the unit
# its inner loop issues.
PIPES = {}


def set_pipes(rates):
    """The ceilings from the measured rates (operations per second)."""
    imad, wide = rates["imad"], rates["imad_wide"]
    PIPES.update({
        "imad": (imad, "IMAD/s (mad.lo.u32, measured)"),
        "imad_wide": (wide, "IMAD.WIDE/s (mad.wide.u32, measured)"),
        "dp4a": (rates["dp4a"], "dp4a/s (measured)"),
        "mad64": (rates["mad64"], "64-bit mad.lo/s (mad.lo.u64, measured)"),
        "mad64x2": (rates["mad64"] / 2, "64x64->128 multiply-adds/s (two 64-bit mads each, measured rate / 2)"),
        "mad64x32": (imad / 3, "64x32-bit multiply-adds/s (three 32-bit multiply-adds each: low and high "
                               "halves of residue x low word half with its carry, residue x high half; measured IMAD / 3)"),
        "dfma": (rates["dfma"], "DFMA/s (fma.rn.f64, measured)"),
        "mma_s8": (rates["mma_s8"], "int8 mma.sync ops/s (m16n8k32, measured)"),
    })


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def tensor_peaks():
    """Dense tensor-core peaks (flops/s) from the measured bf16 rate: fp16 runs
    at the bf16 rate, e4m3 at twice it and e2m1 (block-scaled fp4) at six
    times it (GB300's nominal dense rates 2.25 : 4.5 : 13.5 PFLOP/s; a
    cuBLASLt e4m3 product measured 1.96x bf16 on this GPU)."""
    pk = measured_peaks()
    bf16 = (pk.get("bf16_tflops") or 1900.0) * 1e12
    src = "MEASURED_PEAKS.json bf16_tflops (burst)" if pk.get("bf16_tflops") else "fallback 1.9 PFLOP/s"
    return {"tc_f16": (bf16, "fp16 tcgen05 flops/s (bf16 dense, %s)" % src),
            "tc_f8": (2 * bf16, "e4m3 tcgen05 flops/s (2 x bf16 dense, %s)" % src),
            "tc_e2m1": (6 * bf16, "e2m1 block-scaled tcgen05 flops/s (6 x bf16 dense, %s)" % src),
            "tc_mma_s8": PIPES["mma_s8"]}


def form_roofline(ms: float, work: float, pipe: str = None, peak: float = None, unit: str = None):
    """Achieved rate of `work` units in `ms` against a pipe's ceiling."""
    if pipe is not None:
        peak, unit = PIPES[pipe]
    achieved = work / (ms * 1e-3)
    return {"work_per_launch": work, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": round(achieved / peak, 4)}


def event_time(torch, fn, reps, flush):
    """Median CUDA-event time (ms) of fn over reps calls, L2 flushed before each."""
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
    """Every form on one (A, B); buffers allocated once.  Each form is a list
    of preparation launches, one product launch, and finishing launches, so
    that events can bracket the form and its product kernel separately."""

    def __init__(self, gfp, torch, A, B, tuned):
        self.gfp, self.torch = gfp, torch
        self.A, self.B = A, B
        dev = A.device
        e = lambda *s, dt=torch.uint8: torch.empty(*s, dtype=dt, device=dev)
        g = gfp
        self.forms = {}          # name -> (prep, product, finish, product work, pipe, launches)
        self.outs = {}

        def out(name):
            self.outs[name] = e((M, N))
            return self.outs[name]

        ws = lambda algo: e(max(1, g.gfp_gemm_workspace_size(P, M, K, N, algo)))
        # classical products
        C = out("plain")
        self.forms["plain"] = ([], lambda C=C: g.gfp_gemm(P, A, B, "plain", out=C), [],
                               M * N * K, "imad", 1)
        C, w = out("dp4a"), ws("dp4a")
        self.forms["dp4a"] = ([], lambda C=C, w=w: g.gfp_gemm(P, A, B, "dp4a", out=C, workspace=w), [],
                              M * N * -(-K // 4), "dp4a", 2)
        # Q-adic dot forms: 64-bit words, and the autotuner's choice
        self.dot = {}
        for name, (word, d, Q, kb) in (("dot_u64", ("u64",) + g.gfp_params(P, M, K, N, "dot", "u64")),
                                       ("dot_tuned", tuned)):
            kc = -(-K // (d + 1))
            CA = e((M, kc), dt=g.WORD_DTYPE[word])
            CB = e((kc, N), dt=g.WORD_DTYPE[word])
            C = out(name)
            prep = [lambda CA=CA, word=word, d=d, Q=Q: g.gfp_pack(P, A, d, Q, "rows_rev", word, out=CA),
                    lambda CB=CB, word=word, d=d, Q=Q: g.gfp_pack(P, B, d, Q, "cols", word, out=CB)]
            prod = (lambda CA=CA, CB=CB, C=C, word=word, d=d, Q=Q, kb=kb:
                    g.gfp_gemm_compressed(P, M, K, N, d, Q, "dot", word, CA, CB, out=C, kb=kb))
            pipe = {"u64": "mad64", "u64x128": "mad64x2", "u32w": "imad_wide", "u32": "imad"}[word]
            self.forms[name] = (prep, prod, [], M * N * kc, pipe, 3)
            self.dot[name] = {"word": word, "d_plus_1": d + 1, "t": Q.bit_length() - 1, "kb": kb}
        # right-compressed form with REDQ, then the words unpacked
        dm, Qm, _ = g.gfp_params(P, M, K, N, "mixed", "u64")
        ncm = -(-N // (dm + 1))
        CBr = e((K, ncm), dt=torch.int64)
        CC = e((M, ncm), dt=torch.int64)
        C = out("mixed_u64")
        self.forms["mixed_u64"] = (
            [lambda: g.gfp_pack(P, B, dm, Qm, "rows", "u64", out=CBr)],
            lambda: g.gfp_gemm_compressed(P, M, K, N, dm, Qm, "mixed", "u64", A, CBr, out=CC),
            [lambda C=C: g.gfp_unpack(P, CC, M, N, dm, Qm, "rows", "u64", out=C)],
            M * K * ncm, "mad64x32", 3)
        self.dot["mixed_u64"] = {"word": "u64", "d_plus_1": dm + 1, "t": Qm.bit_length() - 1}
        # exact tensor-core forms (operand conversions inside the call)
        tpk = tensor_peaks()
        launches = {"tc_mma_s8": 3, "tc_f16": 3, "tc_f8": 2, "tc_e2m1": 3}
        for algo in ("tc_mma_s8", "tc_f16", "tc_f8", "tc_e2m1"):
            if algo not in g.ALGOS:
                continue
            C, w = out(algo), ws(algo)
            self.forms[algo] = ([], lambda C=C, w=w, algo=algo: g.gfp_gemm(P, A, B, algo, out=C, workspace=w),
                                [], FLOP, tpk[algo], launches[algo])

    @property
    def products(self):
        return len(self.forms)

    @property
    def launches(self):
        return sum(f[5] for f in self.forms.values())

    def order(self):
        """Forms in the order a step runs them: the tensor-core forms first,
        so that the copies of their results to the host (end to end) overlap
        the long CUDA-core forms, and the copy left after the step is one."""
        tc = [n for n in self.forms if n.startswith("tc_")]
        return tc + [n for n in self.forms if n not in tc]

    def run(self, ev=None, done=None):
        """One step.  ev: name -> four events (form start, product start,
        product end, form end), recorded on the current stream.  done(name),
        if given, is called once the launches completing output `name` are
        issued (to start its copy to the host)."""
        for name in self.order():
            prep, prod, finish = self.forms[name][:3]
            e4 = ev[name] if ev is not None else None
            if e4:
                e4[0].record()
            for f in prep:
                f()
            if e4:
                e4[1].record()
            prod()
            if e4:
                e4[2].record()
            for f in finish:
                f()
            if e4:
                e4[3].record()
            if done is not None:
                done(name)


# ---------------------------------------------------------------------------
# the other workloads (extra keys)
# ---------------------------------------------------------------------------
def fp64_peak(torch):
    """FP64 denominator measured here: cuBLAS DGEMM (torch.matmul in float64)
    at 4096^3, best of 5 (CUDA events).  flops/s."""
    a = torch.rand(4096, 4096, dtype=torch.float64, device="cuda")
    b = torch.rand(4096, 4096, dtype=torch.float64, device="cuda")
    c = torch.empty_like(a)
    for _ in range(2):
        torch.matmul(a, b, out=c)
    best = None
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    return 2.0 * 4096 ** 3 / (best * 1e-3)


def compressed_1024(gfp, torch, inputs, flush, f64_peak):
    """p = 3, m = k = n = 1024: every machine word of the dot form (FP64
    included), the mixed, left and full forms, both classical products and
    the tensor-core forms, each timed alone (median of 7, L2 flushed)."""
    p, m, k, n = 3, 1024, 1024, 1024
    flop = 2.0 * m * n * k
    g = inputs.rng(2, 0)
    A = torch.from_numpy(inputs.residues(g, p, m, k)).cuda()
    B = torch.from_numpy(inputs.residues(g, p, k, n)).cuda()
    dev = A.device
    out = {"workload": "Q-adic compressed GEMM and all forms, p=3, m=k=n=1024, uniform residues"}
    tpk = tensor_peaks()
    pipes = PIPES
    base = {}

    def rec(name, ms, work=None, pipe=None, **extra):
        r = {"ms": round(ms, 5), "value": round(flop / ms / 1e9, 3)}
        for b in ("plain", "dp4a"):
            if b in base:
                r["speedup_vs_" + b] = round(base[b] / ms, 3)
        r.update(extra)
        if work is not None:
            peak, unit = pipes[pipe] if isinstance(pipe, str) else pipe
            r["roofline"] = form_roofline(ms, work, peak=peak, unit=unit)
        out[name] = r

    for algo in ("plain", "dp4a", "tc_mma_s8", "tc_f16", "tc_f8", "tc_e2m1"):
        if algo not in gfp.ALGOS:
            continue
        ws = torch.empty(max(1, gfp.gfp_gemm_workspace_size(p, m, k, n, algo)), dtype=torch.uint8, device=dev)
        C = torch.empty((m, n), dtype=torch.uint8, device=dev)
        ms = event_time(torch, lambda: gfp.gfp_gemm(p, A, B, algo, out=C, workspace=ws), 7, flush)
        work = {"plain": (m * n * k, "imad"), "dp4a": (m * n * -(-k // 4), "dp4a")}.get(algo, (flop, tpk.get(algo)))
        if algo in ("plain", "dp4a"):
            base[algo] = ms
        rec(algo, ms, *work)
    word_pipe = {"u64": "mad64", "u64x128": "mad64x2", "u32w": "imad_wide", "u32": "imad", "f64": "dfma"}
    for word, kb in (("u64", 0), ("u64x128", 0), ("u32w", 0), ("u32", 0), ("f64", 0), ("u32", 60),
                     ("u32w", 140)):
        d, Q, kbr = gfp.gfp_params(p, m, k, n, "dot", word, kb=kb)
        CA = gfp.gfp_pack(p, A, d, Q, "rows_rev", word)
        CB = gfp.gfp_pack(p, B, d, Q, "cols", word)
        C = torch.empty((m, n), dtype=torch.uint8, device=dev)
        t_mm = event_time(torch, lambda: gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "dot", word, CA, CB, out=C,
                                                                 kb=kbr), 7, flush)
        name = "dot_%s" % word + ("_kb%d" % kbr if kbr else "")
        rec(name, t_mm, m * n * -(-k // (d + 1)), word_pipe[word], d_plus_1=d + 1, t=Q.bit_length() - 1, kb=kbr)
    for word in ("u64", "f64"):
        d, Q, _ = gfp.gfp_params(p, m, k, n, "mixed", word)
        CB = gfp.gfp_pack(p, B, d, Q, "rows", word)
        CC = torch.empty((m, -(-n // (d + 1))), dtype=gfp.WORD_DTYPE[word], device=dev)
        ms = event_time(torch, lambda: gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "mixed", word, A, CB, out=CC),
                        7, flush)
        rec("mixed_%s" % word, ms, m * k * -(-n // (d + 1)), "mad64x32" if word == "u64" else "dfma",
            d_plus_1=d + 1, t=Q.bit_length() - 1)
    d, Q, _ = gfp.gfp_params(p, m, k, n, "left", "u64")
    CA = gfp.gfp_pack(p, A, d, Q, "cols", "u64")
    CC = torch.empty((-(-m // (d + 1)), n), dtype=torch.int64, device=dev)
    ms = event_time(torch, lambda: gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "left", "u64", CA, B, out=CC), 7, flush)
    rec("left_u64", ms, -(-m // (d + 1)) * k * n, "mad64x32", d_plus_1=d + 1, t=Q.bit_length() - 1)
    dq, dth, Q = gfp.gfp_params_full(p, m, k, n, "u64")
    CA = gfp.gfp_pack(p, A, dq, Q, "cols", "u64")
    CB = gfp.gfp_pack(p, B, dth, Q ** (dq + 1), "rows", "u64")
    CC = torch.empty((-(-m // (dq + 1)), -(-n // (dth + 1))), dtype=torch.int64, device=dev)
    ms = event_time(torch, lambda: gfp.gfp_gemm_full(p, m, k, n, dq, dth, Q, "u64", CA, CB, out=CC), 7, flush)
    rec("full_u64", ms, -(-m // (dq + 1)) * k * -(-n // (dth + 1)), "mad64", dq=dq, dth=dth, t=Q.bit_length() - 1)
    return out


def tensor_core_8192(gfp, torch, inputs, flush):
    """p in {3, 31, 251}, m = k = n = 8192: every tensor-core algorithm the
    prime allows, median of 5 calls (operand conversion included), with its
    fraction of the dense peak of the pipe it runs on."""
    n = 8192
    flop = 2.0 * n ** 3
    tpk = tensor_peaks()
    out = {"workload": "exact tensor-core GEMM, p in {3,31,251}, m=k=n=8192, uniform residues"}
    for p in (3, 31, 251):
        g = inputs.rng(3, p)
        A = torch.from_numpy(inputs.residues(g, p, n, n)).cuda()
        B = torch.from_numpy(inputs.residues(g, p, n, n)).cuda()
        row = {}
        for algo in ("tc_mma_s8", "tc_f16", "tc_f8", "tc_e2m1"):
            if algo not in gfp.ALGOS or not algo_admits(algo, p):
                continue
            ws = torch.empty(max(1, gfp.gfp_gemm_workspace_size(p, n, n, n, algo)), dtype=torch.uint8,
                             device="cuda")
            C = torch.empty((n, n), dtype=torch.uint8, device="cuda")
            ms = event_time(torch, lambda: gfp.gfp_gemm(p, A, B, algo, out=C, workspace=ws), 5, flush)
            peak, unit = tpk[algo]
            row[algo] = {"ms": round(ms, 4), "value": round(flop / ms / 1e9, 2),
                         "roofline": form_roofline(ms, flop, peak=peak, unit=unit)}
        out["p%d" % p] = row
        del A, B
    return out


def reduce_compress(gfp, torch, inputs, flush):
    """Procedure (compC): the next left operand of a chain A^l, p = 5,
    m = k = n = 16384, 64-bit words.  The dot product followed by a separate
    packing of its residues (two launches, the m n result bytes through HBM)
    against ReduceAndCompress fused into the dot kernel's epilogue (one
    launch); median of 3, L2 flushed."""
    p, n = 5, 16384
    g = inputs.rng(5, 1)
    A = torch.from_numpy(inputs.residues(g, p, n, n)).cuda()
    d, Q, _ = gfp.gfp_params(p, n, n, n, "dot", "u64")
    CA = gfp.gfp_pack(p, A, d, Q, "rows_rev", "u64")
    CB = gfp.gfp_pack(p, A, d, Q, "cols", "u64")
    C = torch.empty((n, n), dtype=torch.uint8, device="cuda")
    W = torch.empty_like(CA)

    def separate():
        gfp.gfp_gemm_compressed(p, n, n, n, d, Q, "dot", "u64", CA, CB, out=C)
        gfp.gfp_pack(p, C, d, Q, "rows_rev", "u64", out=W)

    t_sep = event_time(torch, separate, 3, flush)
    t_fused = event_time(torch, lambda: gfp.gfp_gemm_compressed_compc(p, n, n, n, d, Q, "u64", CA, CB, d, Q, out=W),
                         3, flush)
    flop = 2.0 * n ** 3
    return {"workload": "A^2 mod 5 kept packed as the next left operand, m=k=n=16384, u64 words (d+1=%d)" % (d + 1),
            "separate_ms": round(t_sep, 3), "fused_ms": round(t_fused, 3), "launches_separate": 2,
            "launches_fused": 1, "hbm_bytes_saved": 2 * n * n, "value_fused": round(flop / t_fused / 1e9, 3),
            "unit": UNIT}


def pack_unpack(gfp, torch, A, flush):
    """The conversions of the compressed forms at the headline size (p = 5,
    16384^2, the dot form's u64 words, d+1 = 3): bytes read + written per call
    against the measured HBM copy rate."""
    d, Q, _ = gfp.gfp_params(P, M, K, N, "dot", "u64")
    hbm = (measured_peaks().get("hbm_gbs") or 6800.0) * 1e9
    CA = gfp.gfp_pack(P, A, d, Q, "rows_rev", "u64")
    CB = gfp.gfp_pack(P, A, d, Q, "cols", "u64")
    CR = gfp.gfp_pack(P, A, d, Q, "rows", "u64")
    X = torch.empty_like(A)
    out = {"workload": "p=5, 16384^2 residues <-> u64 words of d+1=%d (t=%d)" % (d + 1, Q.bit_length() - 1)}
    cases = (("pack_rows_rev", lambda: gfp.gfp_pack(P, A, d, Q, "rows_rev", "u64", out=CA), CA),
             ("pack_cols", lambda: gfp.gfp_pack(P, A, d, Q, "cols", "u64", out=CB), CB),
             ("unpack_rows", lambda: gfp.gfp_unpack(P, CR, M, N, d, Q, "rows", "u64", out=X), CR))
    for name, fn, W in cases:
        ms = event_time(torch, fn, 7, flush)
        byts = A.numel() + W.numel() * 8
        out[name] = {"ms": round(ms, 4), "bytes": byts,
                     "roofline": form_roofline(ms, byts, peak=hbm, unit="bytes/s (MEASURED_PEAKS.json hbm_gbs)")}
    return out


def batched_measure(gfp, torch, inputs, flush, flags=0):
    """4096 squares of adjacency matrices in one grouped launch (CUDA graph).
    flags: gfp.PROBLEM_B_IS_A_T declares B = A^T (true here: A symmetric,
    B = A), so that one staged copy of A serves both operands."""
    probs = inputs.batched_problems()
    dev = torch.device("cuda")
    items = []
    flops = 0.0
    for p, A in probs:
        Ad = torch.from_numpy(A).to(dev)
        n = A.shape[0]
        items.append((p, Ad, Ad, torch.empty((n, n), dtype=torch.uint8, device=dev)))
        flops += 2.0 * n ** 3
    arr, cnt = gfp.make_problems(items, flags=flags)
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
    return {"workload": "4096 squares A_i^2 mod p_i of symmetric 0/1 adjacency matrices, n_i log-uniform in "
                        "[16,512], p_i in {3,5,7}", "problems": cnt, "sum_2n3": flops, "ms": round(ms, 4),
            "value": round(flops / ms / 1e9, 3), "unit": UNIT,
            "engines": batched_engines(gfp, table, [A.shape[0] for _, A in probs])}


def algo_admits(algo: str, p: int) -> bool:
    """Primes each tensor-core algorithm takes (include/gfp.h): e2m1 holds the
    centred residues of p <= 7 exactly, e4m3 those of p <= 31."""
    return {"tc_e2m1": p <= 7, "tc_f8": p <= 31}.get(algo, True)


def batched_engines(gfp, table, sizes):
    """The tile kind that ran each size bucket holding problems: the
    autotuner's pick, or the library's default (tcgen05 tiles) where it kept
    the default.  Buckets are by the problem's largest extent."""
    edges = [(32, "n<=32"), (64, "n<=64"), (128, "n<=128"), (256, "n<=256"), (512, "n<=512"),
             (2048, "n<=2048"), (1 << 62, "n>2048")]
    used = {}
    for n in sizes:
        b = next(i for i, (e, _) in enumerate(edges) if n <= e)
        used[b] = used.get(b, 0) + 1
    out = {}
    for b, cnt in sorted(used.items()):
        v = table[b] if b < len(table) else -1
        kind = gfp.BATCHED_KINDS.get(v if v >= 0 else 4, str(v))
        out[edges[b][1]] = {"problems": cnt, "engine": kind, "tuned": v >= 0}
    return out


# ---------------------------------------------------------------------------
# the CPU oracle beside it
# ---------------------------------------------------------------------------
def sample_rows(count):
    """`count` rows of the product spread evenly over m (first and last included)."""
    return np.unique(np.linspace(0, M - 1, count).round().astype(np.int64))


def cpu_oracle_rate(A, B, budget_s=12.0):
    """The oracle (the plain C triple loop over all host cores) on sampled
    rows of the same 16384^3 product, scaled to about budget_s of CPU time."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    rows = sample_rows(cores)
    t0 = time.time()
    oracle.gemm_rows(P, rows, A, B, threads=cores)
    one = time.time() - t0
    count = int(min(1024, max(rows.size, rows.size * budget_s / max(one, 1e-3))))
    rows = sample_rows(count)
    t0 = time.time()
    oracle.gemm_rows(P, rows, A, B, threads=cores)
    per = time.time() - t0
    v = rows.size * 2.0 * K * N / per / 1e12
    return v, cores, "%d of the %d rows of the p=%d %dx%dx%d product (rows spread evenly), %.1f s" % (
        rows.size, M, P, M, K, N, per)


def run_reference(args, rank, world):
    """--impl reference: the oracle as it stands, timed on the host cores on
    --oracle-rows sampled rows of the same product per step."""
    if rank != 0:
        return
    from paper_0803_1975_gb300 import inputs
    import oracle
    oracle.build()
    g = inputs.rng(*SEED)
    A = inputs.residues(g, P, M, K)
    B = inputs.residues(g, P, K, N)
    cores = os.cpu_count() or 1
    rows = sample_rows(args.oracle_rows)
    for _ in range(args.warmup):
        oracle.gemm_rows(P, rows, A, B, threads=cores)
    ts = []
    for _ in range(args.steps):
        t0 = time.time()
        oracle.gemm_rows(P, rows, A, B, threads=cores)
        ts.append(time.time() - t0)
    per = float(np.sum(ts)) / args.steps
    v = rows.size * 2.0 * K * N / per / 1e12
    sample = "%d of the %d rows of the product per step (rows spread evenly)" % (rows.size, M)
    line = {"metric": METRIC, "value": round(v, 5), "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": config_dict(),
            "cpu_baseline": {"value": round(v, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# DRAM bytes (read + written) of one launch of a step kernel, from an ncu
# capture of that kernel on this workload (dram__bytes_read.sum +
# dram__bytes_write.sum); None where no capture of the current kernel exists.
# dot_u64: 17,443,889,920 read + 282,185,472 written, from
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum \
#       --clock-control none -k regex:simt_gemm -c 1 \
#       python -m paper_0803_1975_gb300.run_case --form dot --word u64 --p 5 --size 16384 --reps 1 --warmup 0
# (operands 1.43 GB, result 0.27 GB).
TRAFFIC = {"dot_u64": 17443889920 + 282185472}

KERNEL_NAMES = {"plain": "simt_gemm_kernel<PlainP>", "dp4a": "simt_gemm_kernel<Dp4aT>",
                "dot_u64": "simt_gemm_kernel<DotU64>", "mixed_u64": "simt_gemm_kernel<MixedU64>",
                "tc_mma_s8": "mma_s8_kernel", "tc_f16": "tc_pair_kernel<PairCfg<256, fp16>>",
                "tc_f8": "tc_pair_kernel<PairCfg<256, e4m3>>", "tc_e2m1": "tc_pair_kernel<PairCfg<224, e2m1>>"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gfp", choices=["gfp", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads")
    ap.add_argument("--oracle-rows", type=int, default=ORACLE_ROWS,
                    help="--impl reference: rows of the product the oracle computes per step")
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
    g = inputs.rng(*SEED)
    A_h = inputs.residues(g, P, M, K)
    B_h = inputs.residues(g, P, K, N)
    A = torch.from_numpy(A_h).cuda()
    B = torch.from_numpy(B_h).cuda()
    rates = gfp.gfp_pipe_rates()                        # untimed: measured instruction rates
    set_pipes(rates)
    best, _ = gfp.gfp_dot_autotune(P, M, K, N)          # untimed: word, d, Q, k-block for this shape
    tuned = (best["word"], best["d"], best["Q"], best["kb"])
    step = Step(gfp, torch, A, B, tuned)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        step.run()
    torch.cuda.synchronize()

    # the outputs are the unique product: every form equal, and sampled rows
    # equal to the oracle's (the tests check the full products)
    import oracle
    oracle.build()
    rows = sample_rows(16)
    ref_rows = torch.from_numpy(oracle.gemm_rows(P, rows, A_h, B_h, threads=os.cpu_count() or 1)).cuda()
    first = None
    for name, C in step.outs.items():
        if not torch.equal(C[torch.from_numpy(rows).cuda()], ref_rows):
            raise SystemExit("bench: %s result differs from the oracle" % name)
        if first is not None and not torch.equal(C, first):
            raise SystemExit("bench: %s result differs from %s" % (name, next(iter(step.outs))))
        first = C if first is None else first

    clocks = Clocks(local)
    clocks.start()
    barrier()
    step_ms = []
    form_ms = {n: [] for n in step.forms}
    prod_ms = {n: [] for n in step.forms}
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ev = {n: [torch.cuda.Event(enable_timing=True) for _ in range(4)] for n in step.forms}
        e0.record()
        step.run(ev=ev)
        e1.record()
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for n, e4 in ev.items():
            form_ms[n].append(e4[0].elapsed_time(e4[3]))
            prod_ms[n].append(e4[1].elapsed_time(e4[2]))
    barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(float(np.sum(step_ms)), device="cuda")
    ms_per_step = total_ms / args.steps
    value = world * step.products * FLOP / ms_per_step / 1e9

    # end to end: pinned host inputs -> device -> every form -> results to
    # pinned host memory; each result is copied on a second stream as soon as
    # its form is done (ordered by an event), overlapping the later forms
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
        if not (C.numpy()[rows] == ref_rows.cpu().numpy()).all():
            raise SystemExit("bench: end-to-end %s result differs from the oracle" % k_)

    # each form inside the step; the dominant kernel is the product launch
    # with the largest share of the step
    step_mean = float(np.mean(step_ms))
    f64_peak = fp64_peak(torch) if rank == 0 else None
    forms = {}
    plain_ms = float(np.mean(form_ms["plain"]))
    dp4a_ms = float(np.mean(form_ms["dp4a"]))
    for n, (_, _, _, work, pipe, launches) in step.forms.items():
        fm = float(np.mean(form_ms[n]))
        pm = float(np.mean(prod_ms[n]))
        peak, unit = PIPES[pipe] if isinstance(pipe, str) else pipe
        r = {"ms": round(fm, 3), "value": round(FLOP / fm / 1e9, 3), "kernel_ms": round(pm, 3),
             "speedup_vs_plain": round(plain_ms / fm, 3), "speedup_vs_dp4a": round(dp4a_ms / fm, 3),
             "launches": launches, "share_of_step": round(fm / step_mean, 4),
             "roofline": form_roofline(pm, work, peak=peak, unit=unit)}
        r.update(step.dot.get(n, {}))
        if n in ("tc_f16", "tc_f8", "tc_e2m1") and rates.get("tc_pair_" + n[3:]):
            # cross-check: the dense rate of the same tcgen05 kind on CTA pairs,
            # measured by the library's MMA probe on this GPU (no operand
            # traffic, the full 2.07 GHz clock)
            probe = rates["tc_pair_" + n[3:]]
            r["roofline"]["mma_probe_peak"] = probe
            r["roofline"]["frac_of_mma_probe"] = round(work / (pm * 1e-3) / probe, 4)
        forms[n] = r
    dom = max(step.forms, key=lambda n: np.mean(prod_ms[n]))
    dwork, dpipe = step.forms[dom][3], step.forms[dom][4]
    dpeak, dunit = PIPES[dpipe] if isinstance(dpipe, str) else dpipe
    dms = float(np.mean(prod_ms[dom]))
    tensor = dom.startswith("tc_")
    roofline = {"kernel": KERNEL_NAMES.get(dom, dom) + " (form %s)" % dom,
                "bound": "tensor" if tensor else "alu",
                "achieved": round(dwork / (dms * 1e-3) / 1e12, 4), "peak": round(dpeak / 1e12, 4),
                "unit": "TFLOP/s" if tensor else "T %s" % dunit.split(" (")[0],
                "frac": round(dwork / (dms * 1e-3) / dpeak, 4),
                "peak_source": dunit, "traffic": TRAFFIC.get(dom),
                "launch_ms": round(dms, 4), "work_per_launch": dwork,
                "share_of_step": round(dms / step_mean, 4)}

    extras = {}
    if rank == 0 and not args.no_extras:
        extras["fp64_dgemm_tflops"] = round(f64_peak / 1e12, 4)
        extras["compressed_1024"] = compressed_1024(gfp, torch, inputs, flush, f64_peak)
        extras["tensor_core_8192"] = tensor_core_8192(gfp, torch, inputs, flush)
        extras["reduce_compress"] = reduce_compress(gfp, torch, inputs, flush)
        extras["pack_unpack"] = pack_unpack(gfp, torch, A, flush)
        try:
            extras["batched"] = batched_measure(gfp, torch, inputs, flush)
            sym = batched_measure(gfp, torch, inputs, flush, flags=gfp.PROBLEM_B_IS_A_T)
            extras["batched"]["with_b_is_a_t_flag"] = {k: sym[k] for k in ("ms", "value", "engines")}
        except gfp.GfpError as e:
            extras["batched"] = {"unavailable": str(e)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample = cpu_oracle_rate(A_h, B_h)
        cpu = {"value": round(v, 5), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        peaks = measured_peaks()
        line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u8/u32/u64/f16/e4m3/s8", "data": "synthetic", "config": config_dict(),
                "products_per_step": step.products, "replicas": world,
                "e2e": {"value": round(world * step.products * FLOP / e2e_per / 1e9, 3), "unit": UNIT,
                        "ms_per_step": round(e2e_per, 3),
                        "h2d_bytes_per_step": 2 * M * K, "d2h_bytes_per_step": step.products * M * N},
                "gpu_launches": step.launches * args.steps,
                "roofline": roofline, "forms": forms, "clocks": clk, "cpu_baseline": cpu,
                "pipe_rates": {k: round(v / 1e12, 4) for k, v in rates.items()},
                "measured_peaks": {"hbm_gbs": peaks.get("hbm_gbs"), "bf16_tflops": peaks.get("bf16_tflops")}}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
