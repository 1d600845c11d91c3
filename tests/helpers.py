"""Shared helpers of the GPU tests: building, seeded inputs, cached oracle
results and word-tensor conversion."""
import functools
import os

import numpy as np
import pytest
import torch

import oracle
from paper_0803_1975_gb300 import build as gbuild
from paper_0803_1975_gb300 import gfp, inputs

THREADS = os.cpu_count() or 4


def ensure_built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    gbuild.build()
    oracle.build()
    gfp.load()


def dev(x: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy()


def words_np(t: torch.Tensor, word: str) -> np.ndarray:
    """Word tensor -> numpy array of the words (uint64 / uint32 / float64)."""
    a = host(t)
    if word in ("u64", "u64x128"):
        return a.view(np.uint64)
    if word in ("u32", "u32w"):
        return a.view(np.uint32)
    return a


def np_words_dtype(word: str):
    return {"u64": np.uint64, "u64x128": np.uint64, "u32": np.uint32, "u32w": np.uint32,
            "f64": np.float64}[word]


def to_word_tensor(W: np.ndarray, word: str) -> torch.Tensor:
    if word in ("u64", "u64x128"):
        return dev(W.astype(np.uint64).view(np.int64))
    if word in ("u32", "u32w"):
        return dev(W.astype(np.uint32).view(np.int32))
    return dev(W.astype(np.float64))


@functools.lru_cache(maxsize=64)
def operands(workload: int, trial: int, p: int, m: int, k: int, n: int):
    g = inputs.rng(workload, trial)
    return inputs.residues(g, p, m, k), inputs.residues(g, p, k, n)


@functools.lru_cache(maxsize=64)
def oracle_product(workload: int, trial: int, p: int, m: int, k: int, n: int):
    A, B = operands(workload, trial, p, m, k, n)
    return oracle.gemm(p, A, B, threads=THREADS)


def freivalds(p: int, A: np.ndarray, B: np.ndarray, C: np.ndarray, rounds: int = 8, seed: int = 7):
    """Freivalds' check A (B r) = C r mod p for random r (error <= p^-rounds).
    A property of any correct product, independent of how C was computed."""
    g = np.random.Generator(np.random.PCG64(seed))
    Ai = A.astype(np.int64)
    Bi = B.astype(np.int64)
    Ci = C.astype(np.int64)
    for _ in range(rounds):
        r = g.integers(0, p, size=(B.shape[1], 1), dtype=np.int64)
        lhs = (Ai @ ((Bi @ r) % p)) % p
        rhs = (Ci @ r) % p
        if not (lhs == rhs).all():
            return False
    return True
