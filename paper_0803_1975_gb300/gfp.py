"""Python binding of libgfp (include/gfp.h): argument marshalling only.

Every function here takes torch tensors, passes their device pointers, sizes
and leading dimensions (and the current CUDA stream) to the C-ABI function of
the same name, and raises GfpError on a non-zero status.  All arithmetic runs
in the library's CUDA kernels; there is no other code path.  If libgfp.so has
not been built, the first call raises a RuntimeError naming the build command.

Packed words are returned in tensors of the word's width: torch.int64 for the
64-bit integer words (the bits of the uint64 word), torch.int32 for the
32-bit ones and torch.float64 for FP64 words.
"""
from __future__ import annotations

import ctypes
import os

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgfp.so")
_lib = None

STATUS = {0: "GFP_OK", 1: "GFP_EINVAL", 2: "GFP_EPRIME", 3: "GFP_EBOUND", 4: "GFP_EQ",
          5: "GFP_EUNSUPPORTED", 6: "GFP_ECUDA", 7: "GFP_EWORKSPACE"}
FORMS = {"dot": 0, "mixed": 1, "left": 2}
WORDS = {"u64": 0, "u64x128": 1, "u32w": 2, "u32": 3, "f64": 4}
LAYOUTS = {"rows_rev": 0, "cols": 1, "rows": 2}
ALGOS = {"auto": 0, "plain": 1, "dp4a": 2, "tc_mma_s8": 3, "tc_f16": 4, "dot32": 5, "tc_f8": 6, "tc_e2m1": 7}
BATCHED_KINDS = {0: "hmma64", 1: "hmma32", 2: "dot32", 3: "hmma128", 4: "tcgen05"}
WORD_DTYPE = {"u64": torch.int64, "u64x128": torch.int64, "u32w": torch.int32, "u32": torch.int32,
              "f64": torch.float64}

# Exported names, as declared in include/gfp.h.
EXPORTS = ("gfp_status_string", "gfp_last_cuda_error", "gfp_word_bytes", "gfp_params", "gfp_pack",
           "gfp_unpack", "gfp_gemm_workspace_size", "gfp_gemm", "gfp_gemm_compressed",
           "gfp_batched_workspace_size", "gfp_gemm_batched", "gfp_batched_prepare",
           "gfp_batched_launch", "gfp_batched_autotune", "gfp_batched_set_table",
           "gfp_gemm_noalloc", "gfp_gemm_full", "gfp_params_full", "gfp_pack_block",
           "gfp_unpack_block", "gfp_params_vb", "gfp_pack_vb", "gfp_gemm_compressed_vb", "gfp_amax",
           "gfp_winograd_workspace_size", "gfp_gemm_compressed_winograd", "gfp_dot_autotune_workspace_size",
           "gfp_dot_autotune", "gfp_selftest_wait_limit", "gfp_pipe_rates", "gfp_gemm_compressed_compc")


class GfpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        name = STATUS.get(status, str(status))
        msg = "%s failed: %s" % (where, name)
        if status == 6 and _lib is not None:
            msg += " (cudaError %d)" % _lib.gfp_last_cuda_error()
        super().__init__(msg)


class DotChoice(ctypes.Structure):
    """struct gfp_dot_choice."""
    _fields_ = [("word", ctypes.c_int32), ("d", ctypes.c_int32), ("Q", ctypes.c_uint64), ("kb", ctypes.c_int64),
                ("ms", ctypes.c_float), ("reserved", ctypes.c_int32)]


class Problem(ctypes.Structure):
    """struct gfp_problem."""
    _fields_ = [("p", ctypes.c_uint32), ("m", ctypes.c_int32), ("k", ctypes.c_int32),
                ("n", ctypes.c_int32), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
                ("C", ctypes.c_void_p), ("lda", ctypes.c_int32), ("ldb", ctypes.c_int32),
                ("ldc", ctypes.c_int32), ("flags", ctypes.c_int32)]


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libgfp.so (once) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError("libgfp.so is not built (%s); run `python -m paper_0803_1975_gb300.build` "
                           "or __graft_entry__.build()" % _LIB_PATH)
    L = ctypes.CDLL(_LIB_PATH)
    i64, u32, u64, vp, ip = ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
    st = ctypes.c_int
    L.gfp_status_string.argtypes = [st]
    L.gfp_status_string.restype = ctypes.c_char_p
    L.gfp_last_cuda_error.argtypes = []
    L.gfp_last_cuda_error.restype = ip
    L.gfp_word_bytes.argtypes = [ip]
    L.gfp_word_bytes.restype = ctypes.c_size_t
    L.gfp_params.argtypes = [u32, i64, i64, i64, ip, ip, ctypes.POINTER(ip), ctypes.POINTER(u64),
                             ctypes.POINTER(i64)]
    L.gfp_params.restype = st
    L.gfp_pack.argtypes = [u32, i64, i64, vp, i64, ip, u64, ip, ip, vp, i64, vp]
    L.gfp_pack.restype = st
    L.gfp_params_vb.argtypes = [u32, i64, i64, i64, ip, ip, u32, u32, ctypes.POINTER(ip), ctypes.POINTER(u64),
                                ctypes.POINTER(i64)]
    L.gfp_params_vb.restype = st
    L.gfp_pack_vb.argtypes = [u32, u32, i64, i64, vp, i64, ip, u64, ip, ip, vp, i64, vp]
    L.gfp_pack_vb.restype = st
    L.gfp_gemm_compressed_vb.argtypes = [u32, i64, i64, i64, ip, u64, ip, ip, u32, u32, vp, i64, vp, i64, vp,
                                         i64, i64, vp]
    L.gfp_gemm_compressed_vb.restype = st
    L.gfp_amax.argtypes = [i64, i64, vp, i64, vp, vp]
    L.gfp_amax.restype = st
    L.gfp_dot_autotune_workspace_size.argtypes = [i64, i64, i64, ctypes.POINTER(ctypes.c_size_t)]
    L.gfp_dot_autotune_workspace_size.restype = st
    L.gfp_dot_autotune.argtypes = [u32, i64, i64, i64, vp, ctypes.c_size_t, vp, ctypes.POINTER(DotChoice),
                                   ctypes.POINTER(DotChoice), ip, ctypes.POINTER(ip)]
    L.gfp_dot_autotune.restype = st
    L.gfp_selftest_wait_limit.argtypes = [vp, ctypes.c_size_t, u32, ctypes.POINTER(ip), vp]
    L.gfp_selftest_wait_limit.restype = st
    L.gfp_pipe_rates.argtypes = [ctypes.POINTER(ctypes.c_double), ip, vp, ctypes.c_size_t, vp]
    L.gfp_pipe_rates.restype = st
    L.gfp_gemm_compressed_compc.argtypes = [u32, i64, i64, i64, ip, u64, ip, vp, i64, vp, i64, i64, ip, u64, vp,
                                            i64, vp]
    L.gfp_gemm_compressed_compc.restype = st
    L.gfp_winograd_workspace_size.argtypes = [i64, i64, i64, ip, ip, ctypes.POINTER(ctypes.c_size_t)]
    L.gfp_winograd_workspace_size.restype = st
    L.gfp_gemm_compressed_winograd.argtypes = [u32, i64, i64, i64, ip, u64, vp, i64, vp, i64, vp, i64, ip, vp,
                                               ctypes.c_size_t, vp]
    L.gfp_gemm_compressed_winograd.restype = st
    L.gfp_unpack.argtypes = [u32, i64, i64, vp, i64, ip, u64, ip, ip, vp, i64, vp]
    L.gfp_unpack.restype = st
    L.gfp_gemm_workspace_size.argtypes = [u32, i64, i64, i64, ip, ctypes.POINTER(ctypes.c_size_t)]
    L.gfp_gemm_workspace_size.restype = st
    L.gfp_gemm.argtypes = [u32, i64, i64, i64, vp, i64, vp, i64, vp, i64, ip, vp, ctypes.c_size_t, vp]
    L.gfp_gemm.restype = st
    L.gfp_gemm_compressed.argtypes = [u32, i64, i64, i64, ip, u64, ip, ip, vp, i64, vp, i64, vp, i64,
                                      i64, vp]
    L.gfp_gemm_compressed.restype = st
    L.gfp_gemm_full.argtypes = [u32, i64, i64, i64, ip, ip, u64, ip, vp, i64, vp, i64, vp, i64, vp]
    L.gfp_gemm_full.restype = st
    L.gfp_params_full.argtypes = [u32, i64, i64, i64, ip, ctypes.POINTER(ip), ctypes.POINTER(ip),
                                  ctypes.POINTER(u64)]
    L.gfp_params_full.restype = st
    for name in ("gfp_pack_block", "gfp_unpack_block"):
        f = getattr(L, name)
        f.argtypes = [u32, i64, i64, vp, i64, ip, ip, u64, ip, vp, i64, vp]
        f.restype = st
    L.gfp_gemm_noalloc.argtypes = [u32, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp]
    L.gfp_gemm_noalloc.restype = st
    L.gfp_batched_workspace_size.argtypes = [i64, ctypes.POINTER(Problem), ctypes.POINTER(ctypes.c_size_t)]
    L.gfp_batched_workspace_size.restype = st
    for name in ("gfp_gemm_batched", "gfp_batched_prepare"):
        f = getattr(L, name)
        f.argtypes = [i64, ctypes.POINTER(Problem), ip, ctypes.POINTER(st), vp, ctypes.c_size_t, vp]
        f.restype = st
    L.gfp_batched_launch.argtypes = [vp, ctypes.c_size_t, vp]
    L.gfp_batched_launch.restype = st
    L.gfp_batched_autotune.argtypes = [i64, ctypes.POINTER(Problem), vp, ctypes.c_size_t, vp,
                                       ctypes.POINTER(ip), ip]
    L.gfp_batched_autotune.restype = st
    L.gfp_batched_set_table.argtypes = [ctypes.POINTER(ip), ip]
    L.gfp_batched_set_table.restype = st
    _lib = L
    return L


def _check(status: int, where: str):
    if status != 0:
        raise GfpError(status, where)


def _stream(t: torch.Tensor | None = None, stream=None):
    if stream is not None:
        return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    dev = t.device if t is not None else None
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _mat(t: torch.Tensor, dtype, name: str):
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    # the column stride matters only when a row holds more than one entry
    if t.dim() != 2 or not t.is_cuda or (t.numel() > 0 and t.shape[1] > 1 and t.stride(1) != 1):
        raise ValueError("%s must be a 2-D CUDA tensor with unit column stride" % name)
    return ctypes.c_void_p(t.data_ptr()), max(t.stride(0), t.shape[1], 1)


def cdiv(a: int, b: int) -> int:
    return -(-a // b)


# ----------------------------------------------------------------------------
def gfp_params(p: int, m: int, k: int, n: int, form: str = "dot", word: str = "u64",
               d: int | None = None, Q: int | None = None, kb: int = 0):
    """Choose (d is None) or validate (d, Q, kb).  Returns (d, Q, kb)."""
    L = load()
    dd = ctypes.c_int(-1 if d is None else d)
    QQ = ctypes.c_uint64(0 if Q is None else Q)
    kk = ctypes.c_int64(kb)
    _check(L.gfp_params(p, m, k, n, FORMS[form], WORDS[word], ctypes.byref(dd), ctypes.byref(QQ),
                        ctypes.byref(kk)), "gfp_params")
    return dd.value, QQ.value, kk.value


def gfp_params_vb(p: int, m: int, k: int, n: int, amax_a: int, amax_b: int, form: str = "dot",
                  word: str = "u64", d: int | None = None, Q: int | None = None, kb: int = 0):
    """gfp_params with entries of A at most amax_a and of B at most amax_b."""
    L = load()
    dd = ctypes.c_int(-1 if d is None else d)
    QQ = ctypes.c_uint64(0 if Q is None else Q)
    kk = ctypes.c_int64(kb)
    _check(L.gfp_params_vb(p, m, k, n, FORMS[form], WORDS[word], amax_a, amax_b, ctypes.byref(dd),
                           ctypes.byref(QQ), ctypes.byref(kk)), "gfp_params_vb")
    return dd.value, QQ.value, kk.value


def gfp_amax(X: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Largest entry of a uint8 matrix, as a one-element int32 CUDA tensor
    (written asynchronously)."""
    L = load()
    rows, cols = X.shape
    if out is None:
        out = torch.empty(1, dtype=torch.int32, device=X.device)
    xp, ldx = _mat(X, torch.uint8, "X")
    _check(L.gfp_amax(rows, cols, xp, ldx, out.data_ptr(), _stream(X, stream)), "gfp_amax")
    return out


def packed_shape(layout: str, rows: int, cols: int, d: int):
    if layout == "cols":
        return cdiv(rows, d + 1), cols
    return rows, cdiv(cols, d + 1)


def gfp_pack(p: int, X: torch.Tensor, d: int, Q: int, layout: str, word: str = "u64",
             out: torch.Tensor | None = None, stream=None, amax: int | None = None) -> torch.Tensor:
    """Pack X; with amax (<= p - 1) the word bounds of gfp_pack_vb apply."""
    L = load()
    rows, cols = X.shape
    wr, wc = packed_shape(layout, rows, cols, d)
    if out is None:
        out = torch.empty((wr, wc), dtype=WORD_DTYPE[word], device=X.device)
    xp, ldx = _mat(X, torch.uint8, "X")
    wp, ldw = _mat(out, WORD_DTYPE[word], "W")
    if amax is None:
        _check(L.gfp_pack(p, rows, cols, xp, ldx, d, Q, LAYOUTS[layout], WORDS[word], wp, ldw,
                          _stream(X, stream)), "gfp_pack")
    else:
        _check(L.gfp_pack_vb(p, amax, rows, cols, xp, ldx, d, Q, LAYOUTS[layout], WORDS[word], wp, ldw,
                             _stream(X, stream)), "gfp_pack_vb")
    return out


def gfp_unpack(p: int, W: torch.Tensor, rows: int, cols: int, d: int, Q: int, layout: str,
               word: str = "u64", out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    L = load()
    if out is None:
        out = torch.empty((rows, cols), dtype=torch.uint8, device=W.device)
    wp, ldw = _mat(W, WORD_DTYPE[word], "W")
    xp, ldx = _mat(out, torch.uint8, "X")
    _check(L.gfp_unpack(p, rows, cols, wp, ldw, d, Q, LAYOUTS[layout], WORDS[word], xp, ldx,
                        _stream(W, stream)), "gfp_unpack")
    return out


def gfp_gemm_workspace_size(p: int, m: int, k: int, n: int, algo: str = "auto") -> int:
    L = load()
    b = ctypes.c_size_t(0)
    _check(L.gfp_gemm_workspace_size(p, m, k, n, ALGOS[algo], ctypes.byref(b)),
           "gfp_gemm_workspace_size")
    return b.value


def gfp_gemm(p: int, A: torch.Tensor, B: torch.Tensor, algo: str = "auto",
             out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
             stream=None) -> torch.Tensor:
    L = load()
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    if out is None:
        out = torch.empty((m, n), dtype=torch.uint8, device=A.device)
    need = gfp_gemm_workspace_size(p, m, k, n, algo)
    if need and workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=A.device)
    ap, lda = _mat(A, torch.uint8, "A")
    bp, ldb = _mat(B, torch.uint8, "B")
    cp, ldc = _mat(out, torch.uint8, "C")
    ws = ctypes.c_void_p(workspace.data_ptr() if workspace is not None else 0)
    wsb = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(L.gfp_gemm(p, m, k, n, ap, lda, bp, ldb, cp, ldc, ALGOS[algo], ws, wsb,
                      _stream(A, stream)), "gfp_gemm")
    return out


def gfp_params_full(p: int, m: int, k: int, n: int, word: str = "u64", dq: int | None = None,
                    dth: int = 0, Q: int = 0):
    """Choose (dq is None) or validate the (dq, dth, Q) of full compression."""
    L = load()
    a = ctypes.c_int(-1 if dq is None else dq)
    b = ctypes.c_int(dth)
    q = ctypes.c_uint64(Q)
    _check(L.gfp_params_full(p, m, k, n, WORDS[word], ctypes.byref(a), ctypes.byref(b), ctypes.byref(q)),
           "gfp_params_full")
    return a.value, b.value, q.value


def gfp_pack_block(p: int, X: torch.Tensor, dq: int, dth: int, Q: int, word: str = "u64",
                   out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    L = load()
    rows, cols = X.shape
    if out is None:
        out = torch.empty((cdiv(rows, dq + 1), cdiv(cols, dth + 1)), dtype=WORD_DTYPE[word], device=X.device)
    xp, ldx = _mat(X, torch.uint8, "X")
    wp, ldw = _mat(out, WORD_DTYPE[word], "W")
    _check(L.gfp_pack_block(p, rows, cols, xp, ldx, dq, dth, Q, WORDS[word], wp, ldw, _stream(X, stream)),
           "gfp_pack_block")
    return out


def gfp_unpack_block(p: int, W: torch.Tensor, rows: int, cols: int, dq: int, dth: int, Q: int,
                     word: str = "u64", out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    L = load()
    if out is None:
        out = torch.empty((rows, cols), dtype=torch.uint8, device=W.device)
    wp, ldw = _mat(W, WORD_DTYPE[word], "W")
    xp, ldx = _mat(out, torch.uint8, "X")
    _check(L.gfp_unpack_block(p, rows, cols, wp, ldw, dq, dth, Q, WORDS[word], xp, ldx, _stream(W, stream)),
           "gfp_unpack_block")
    return out


def gfp_gemm_full(p: int, m: int, k: int, n: int, dq: int, dth: int, Q: int, word: str,
                  CA: torch.Tensor, CB: torch.Tensor, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """Section 4: CA (COLS of A, base Q) x CB (ROWS of B, base Q^(dq+1)) -> CC
    words in the block layout."""
    L = load()
    wdt = WORD_DTYPE[word]
    if out is None:
        out = torch.empty((cdiv(m, dq + 1), cdiv(n, dth + 1)), dtype=wdt, device=CB.device)
    ap, lda = _mat(CA, wdt, "CA")
    bp, ldb = _mat(CB, wdt, "CB")
    cp, ldc = _mat(out, wdt, "CC")
    _check(L.gfp_gemm_full(p, m, k, n, dq, dth, Q, WORDS[word], ap, lda, bp, ldb, cp, ldc,
                           _stream(CB, stream)), "gfp_gemm_full")
    return out


def gfp_gemm_noalloc(p: int, A: torch.Tensor, B: torch.Tensor, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    """gfp_gemm(..., 'tc_mma_s8') without a workspace, for callers that may not
    allocate device memory at call time (the output, if not given, is
    allocated here by torch before the call)."""
    L = load()
    m, k = A.shape
    n = B.shape[1]
    if out is None:
        out = torch.empty((m, n), dtype=torch.uint8, device=A.device)
    ap, lda = _mat(A, torch.uint8, "A")
    bp, ldb = _mat(B, torch.uint8, "B")
    cp, ldc = _mat(out, torch.uint8, "C")
    _check(L.gfp_gemm_noalloc(p, m, k, n, ap, lda, bp, ldb, cp, ldc, _stream(A, stream)),
           "gfp_gemm_noalloc")
    return out


def gfp_gemm_compressed(p: int, m: int, k: int, n: int, d: int, Q: int, form: str, word: str,
                        CA_or_A: torch.Tensor, CB: torch.Tensor, out: torch.Tensor | None = None,
                        kb: int = 0, stream=None, amax=None) -> torch.Tensor:
    """form 'dot': CA (ROWS_REV words) x CB (COLS words) -> uint8 C (m x n).
    form 'mixed': uint8 A x CB (ROWS words) -> CC words (m x ceil(n/(d+1))).
    amax = (amax_a, amax_b): validate against the value-aware bound
    (gfp_gemm_compressed_vb)."""
    L = load()
    if amax is not None:
        va, vb = amax
        fn = lambda *a: L.gfp_gemm_compressed_vb(*a[:8], va, vb, *a[8:])
    else:
        fn = L.gfp_gemm_compressed
    wdt = WORD_DTYPE[word]
    if form == "dot":
        ap, lda = _mat(CA_or_A, wdt, "CA")
        if out is None:
            out = torch.empty((m, n), dtype=torch.uint8, device=CB.device)
        cp, ldc = _mat(out, torch.uint8, "C")
    elif form == "left":
        ap, lda = _mat(CA_or_A, wdt, "CA")
        if out is None:
            out = torch.empty((cdiv(m, d + 1), n), dtype=wdt, device=CB.device)
        cp, ldc = _mat(out, wdt, "CC")
        bp, ldb = _mat(CB, torch.uint8, "B")
        _check(fn(p, m, k, n, d, Q, FORMS[form], WORDS[word], ap, lda, bp, ldb, cp,
                  ldc, kb, _stream(CB, stream)), "gfp_gemm_compressed")
        return out
    else:
        ap, lda = _mat(CA_or_A, torch.uint8, "A")
        if out is None:
            out = torch.empty((m, cdiv(n, d + 1)), dtype=wdt, device=CB.device)
        cp, ldc = _mat(out, wdt, "CC")
    bp, ldb = _mat(CB, wdt, "CB")
    _check(fn(p, m, k, n, d, Q, FORMS[form], WORDS[word], ap, lda, bp, ldb, cp,
              ldc, kb, _stream(CB, stream)), "gfp_gemm_compressed")
    return out


WORD_NAMES = {v: k for k, v in WORDS.items()}


def gfp_dot_autotune(p: int, m: int, k: int, n: int, device=None, stream=None):
    """Fastest (word, d, Q, kb) of the dot form for (p, m, k, n) on this GPU.
    Returns (best, all): dicts with word, d, Q, kb, ms."""
    L = load()
    need = ctypes.c_size_t(0)
    _check(L.gfp_dot_autotune_workspace_size(m, k, n, ctypes.byref(need)), "gfp_dot_autotune_workspace_size")
    dev = torch.device("cuda") if device is None else device
    ws = torch.empty(max(need.value, 1), dtype=torch.uint8, device=dev)
    best = DotChoice()
    arr = (DotChoice * 128)()
    cnt = ctypes.c_int(0)
    _check(L.gfp_dot_autotune(p, m, k, n, ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(ws, stream),
                              ctypes.byref(best), arr, 128, ctypes.byref(cnt)), "gfp_dot_autotune")
    conv = lambda c: {"word": WORD_NAMES[c.word], "d": c.d, "Q": c.Q, "kb": c.kb, "ms": c.ms}
    return conv(best), [conv(arr[i]) for i in range(min(cnt.value, 128))]


def gfp_selftest_wait_limit(limit_ms: int = 100, device=None, stream=None) -> int:
    """Run the bounded-wait self-test; returns the kernel's status word."""
    L = load()
    dev = torch.device("cuda") if device is None else device
    ws = torch.empty(82176, dtype=torch.uint8, device=dev)
    out = ctypes.c_int(0)
    _check(L.gfp_selftest_wait_limit(ctypes.c_void_p(ws.data_ptr()), ws.numel(), limit_ms, ctypes.byref(out),
                                     _stream(ws, stream)), "gfp_selftest_wait_limit")
    return out.value


def gfp_gemm_compressed_compc(p: int, m: int, k: int, n: int, d: int, Q: int, word: str, CA: torch.Tensor,
                              CB: torch.Tensor, d_out: int, Q_out: int, kb: int = 0,
                              out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """ReduceAndCompress fused into the dot form: the residues of CA x CB
    (gfp_gemm_compressed(dot, word)) as reversed-row words of (d_out, Q_out).
    Returns (or fills) an m x ceil(n/(d_out+1)) tensor of words."""
    L = load()
    dt = WORD_DTYPE[word]
    if out is None:
        out = torch.empty((m, cdiv(n, d_out + 1)), dtype=dt, device=CA.device)
    ap, lda = _mat(CA, dt, "CA")
    bp, ldb = _mat(CB, dt, "CB")
    cp, ldc = _mat(out, dt, "out")
    _check(L.gfp_gemm_compressed_compc(p, m, k, n, d, Q, WORDS[word], ap, lda, bp, ldb, kb, d_out, Q_out,
                                       cp, ldc, _stream(out, stream)),
           "gfp_gemm_compressed_compc")
    return out


PIPE_RATES = ("imad", "imad_wide", "mad64", "dp4a", "dfma", "mma_s8", "tc_f16", "tc_f8", "tc_e2m1",
              "tc_e2m1_nvf4", "tc_pair_f16", "tc_pair_f8", "tc_pair_e2m1")


def gfp_pipe_rates(device=None, stream=None) -> dict:
    """Measured instruction rates (operations per second) of the current GPU:
    {"imad", "imad_wide", "mad64", "dp4a", "dfma", "mma_s8"} in operations per
    second and {"tc_f16", "tc_f8", "tc_e2m1", "tc_e2m1_nvf4", "tc_pair_f16",
    "tc_pair_f8", "tc_pair_e2m1"} (dense tcgen05 rates) in flops
    per second."""
    L = load()
    ws = torch.empty(256, dtype=torch.uint8, device=device or "cuda")
    out = (ctypes.c_double * len(PIPE_RATES))()
    _check(L.gfp_pipe_rates(out, len(PIPE_RATES), ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(ws, stream)),
           "gfp_pipe_rates")
    return dict(zip(PIPE_RATES, list(out)))


def gfp_winograd_workspace_size(m: int, k: int, n: int, d: int, levels: int) -> int:
    L = load()
    out = ctypes.c_size_t(0)
    _check(L.gfp_winograd_workspace_size(m, k, n, d, levels, ctypes.byref(out)), "gfp_winograd_workspace_size")
    return out.value


def gfp_gemm_compressed_winograd(p: int, m: int, k: int, n: int, d: int, Q: int, CA: torch.Tensor,
                                 CB: torch.Tensor, levels: int = 1, out: torch.Tensor | None = None,
                                 workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Dot form in 64-bit words with `levels` levels of Strassen-Winograd
    over Z/2^64 on the words: CA (ROWS_REV) x CB (COLS) -> uint8 C (m x n)."""
    L = load()
    ap, lda = _mat(CA, torch.int64, "CA")
    bp, ldb = _mat(CB, torch.int64, "CB")
    if out is None:
        out = torch.empty((m, n), dtype=torch.uint8, device=CB.device)
    cp, ldc = _mat(out, torch.uint8, "C")
    need = gfp_winograd_workspace_size(m, k, n, d, levels)
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=CB.device)
    _check(L.gfp_gemm_compressed_winograd(p, m, k, n, d, Q, ap, lda, bp, ldb, cp, ldc, levels,
                                          ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                          _stream(CB, stream)), "gfp_gemm_compressed_winograd")
    return out


PROBLEM_B_IS_A_T = 1      # GFP_PROBLEM_B_IS_A_T


def make_problems(items, flags: int = 0) -> ctypes.Array:
    """items: iterable of (p, A, B, C) CUDA uint8 tensors -> gfp_problem array;
    `flags` (e.g. PROBLEM_B_IS_A_T) is set on every problem."""
    items = list(items)
    arr = (Problem * max(len(items), 1))()
    for i, (p, A, B, C) in enumerate(items):
        m, k = A.shape
        n = B.shape[1]
        # leading dimensions as _mat reads them (a one-row view's stride(0) is arbitrary)
        lds = [_mat(X, torch.uint8, name)[1] for X, name in ((A, "A"), (B, "B"), (C, "C"))]
        arr[i] = Problem(p, m, k, n, A.data_ptr(), B.data_ptr(), C.data_ptr(), *lds, flags)
    return arr, len(items)


def gfp_batched_workspace_size(probs, count: int) -> int:
    L = load()
    b = ctypes.c_size_t(0)
    _check(L.gfp_batched_workspace_size(count, probs, ctypes.byref(b)), "gfp_batched_workspace_size")
    return b.value


def gfp_gemm_batched(probs, count: int, algo: str = "auto", workspace: torch.Tensor | None = None,
                     device=None, stream=None, statuses: bool = False):
    """probs/count from make_problems().  Returns the workspace (and the
    per-problem statuses when asked)."""
    L = load()
    need = gfp_batched_workspace_size(probs, count)
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=device or "cuda")
    st = (ctypes.c_int * max(count, 1))()
    r = L.gfp_gemm_batched(count, probs, ALGOS[algo], st, ctypes.c_void_p(workspace.data_ptr()),
                           workspace.numel(), _stream(workspace, stream))
    if statuses:
        return workspace, r, list(st[:count])
    _check(r, "gfp_gemm_batched")
    return workspace


def gfp_batched_prepare(probs, count: int, algo: str, workspace: torch.Tensor, stream=None):
    L = load()
    st = (ctypes.c_int * max(count, 1))()
    _check(L.gfp_batched_prepare(count, probs, ALGOS[algo], st, ctypes.c_void_p(workspace.data_ptr()),
                                 workspace.numel(), _stream(workspace, stream)), "gfp_batched_prepare")


def gfp_batched_launch(workspace: torch.Tensor, stream=None):
    L = load()
    _check(L.gfp_batched_launch(ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                _stream(workspace, stream)), "gfp_batched_launch")


def gfp_batched_autotune(probs, count: int, workspace: torch.Tensor | None = None, device=None,
                         stream=None):
    """Time each tile kind per size bucket on these problems; the library keeps
    the fastest for GFP_ALGO_AUTO.  Returns the table (kind index or -1 per
    bucket)."""
    L = load()
    if workspace is None:
        workspace = torch.empty(max(gfp_batched_workspace_size(probs, count), 1), dtype=torch.uint8,
                                device=device or "cuda")
    table = (ctypes.c_int * 7)()
    _check(L.gfp_batched_autotune(count, probs, ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                  _stream(workspace, stream), table, 7), "gfp_batched_autotune")
    return list(table)


def gfp_batched_set_table(table):
    L = load()
    arr = (ctypes.c_int * len(table))(*table)
    _check(L.gfp_batched_set_table(arr, len(table)), "gfp_batched_set_table")
