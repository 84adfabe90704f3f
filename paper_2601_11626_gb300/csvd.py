"""Thin ctypes binding of the csvd C ABI (``include/csvd.h``).

Argument marshalling only: torch tensors supply device memory and the
current CUDA stream; every step of the computation runs in the library's
kernels.  There is no CPU fallback: ``lib()`` raises when the CUDA library
is missing or no GPU is present.
"""
from __future__ import annotations

import ctypes as C
import math
import enum
import os

import numpy as np
import torch

from . import _build

_LIB = None


class Status(enum.IntEnum):
    OK = 0
    ERR_ARG = 1
    ERR_SHAPE = 2
    ERR_CUDA = 3
    ERR_OOM = 4
    ERR_NOT_CONVERGED = 5
    ERR_TIMEOUT = 6
    ERR_UNIMPLEMENTED = 7


PLAIN, MIXED, GRAM_FP32 = 0, 1, 2
PRECISION = {"plain": PLAIN, "mixed": MIXED, "gram_fp32": GRAM_FP32}


def _prec(precision: str) -> int:
    """C enum of a precision name: "plain" (residual + Jacobi, FP32 SIMT),
    "mixed" (tensor-core Gram route) or "gram_fp32" (the Gram route with
    FP32 SIMT products)."""
    try:
        return PRECISION[precision]
    except KeyError:
        raise ValueError(f"precision must be one of {sorted(PRECISION)}, not {precision!r}")
ALGO = {"weyl": 1, "residual": 2, "approx": 3}
SORT = {"frobenius": 0, "residual": 1}
F32, BF16 = 0, 1


class CsvdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"csvd: {Status(status).name}: {msg}")
        self.status = Status(status)


class Block(C.Structure):
    _fields_ = [("ptr", C.c_void_p), ("k", C.c_int64), ("ld", C.c_int64),
                ("dtype", C.c_int32), ("reserved", C.c_int32)]


def _sig(lib):
    P, I32, I64, D, VP = C.POINTER, C.c_int32, C.c_int64, C.c_double, C.c_void_p
    lib.csvd_last_error.restype = C.c_char_p
    lib.csvd_version.restype = C.c_char_p
    lib.csvd_incr_init.argtypes = [P(VP), I64, I32, I32, VP]
    lib.csvd_incr_append.argtypes = [VP, P(Block)]
    lib.csvd_incr_sigma.argtypes = [VP, P(C.c_float), P(I32)]
    lib.csvd_incr_load.argtypes = [VP, VP, I64, I32, P(C.c_float), D, D]
    lib.csvd_gram_apply.argtypes = [VP, I64, I64, I32, P(Block), I32, VP, I64, VP]
    lib.csvd_reconstruct.argtypes = [VP, I64, VP, I64, I32, P(Block), I32, VP, I64, VP, I64, VP,
                                     P(D), P(D)]
    lib.csvd_incr_basis.argtypes = [VP, VP, I64]
    lib.csvd_tail_error.argtypes = [VP, P(D), P(D), P(D), P(D)]
    lib.csvd_incr_free.argtypes = [VP]
    lib.csvd_score.argtypes = [P(VP), I32, P(I32), P(Block), I32, D, I32, VP, I64, VP, VP, VP]
    lib.csvd_score_plan.argtypes = [P(VP), I32, P(I32), P(Block), I32, D, I32, VP, I64, VP, VP, VP,
                                    P(VP)]
    lib.csvd_plan_launch.argtypes = [VP, VP]
    lib.csvd_plan_status.argtypes = [VP, VP]
    lib.csvd_plan_free.argtypes = [VP]
    lib.csvd_score_columns.argtypes = [P(VP), I32, P(I32), VP, I64, I32, D, VP, I64, VP, VP, VP]
    lib.csvd_stream_init.argtypes = [P(VP), I64, I32, D, I32, VP]
    lib.csvd_stream_push.argtypes = [VP, P(Block), P(I32), P(D), P(D)]
    lib.csvd_stream_count.argtypes = [VP, P(I32)]
    lib.csvd_stream_cluster.argtypes = [VP, I32, P(VP), P(I32)]
    lib.csvd_stream_free.argtypes = [VP]
    lib.csvd_bounds.argtypes = [P(Block), I32, I64, I32, VP, P(D), P(D), P(D), P(D)]
    lib.csvd_cluster.argtypes = [P(Block), I32, I64, I32, D, I32, I32, I32, VP, P(I32), P(D),
                                 P(D), P(D)]
    lib.csvd_tail_grad.argtypes = [VP, I64, I64, I32, P(Block), P(Block), I32, D, VP]
    lib.csvd_block_energy.argtypes = [P(Block), I32, I64, VP, P(D)]
    lib.csvd_set_allocator.argtypes = [VP, VP, VP]
    lib.csvd_debug_limits.argtypes = [I32, I32, I64, I32]
    lib.csvd_tune_set.argtypes = [I32, I32]
    lib.csvd_tail_energy.argtypes = [VP, I64, I64, I32, P(Block), I32, VP, P(D)]
    lib.csvd_top_basis.argtypes = [P(Block), I32, I64, I32, I32, I32, VP, VP, I64, P(I32)]
    lib.csvd_randomized_tail.argtypes = [P(Block), P(VP), I32, I64, I32, I32, I32, VP, P(D), VP,
                                         I64]
    lib.csvd_tune_get.argtypes = [P(I32), P(I32)]
    lib.csvd_score_one_noalloc.argtypes = [VP, P(Block), D, VP, VP, VP, VP]
    lib.csvd_score_one_noalloc.restype = C.c_int
    lib.csvd_launch_count.restype = C.c_int64
    lib.csvd_profile.argtypes = [I32]
    lib.csvd_profile.restype = C.c_int
    lib.csvd_profile_report.argtypes = [C.c_char_p, I64]
    lib.csvd_profile_report.restype = C.c_int
    for name in ("csvd_incr_init", "csvd_incr_append", "csvd_incr_sigma", "csvd_incr_basis",
                 "csvd_incr_load", "csvd_gram_apply",
                 "csvd_tail_error", "csvd_incr_free", "csvd_score", "csvd_score_columns", "csvd_bounds",
                 "csvd_stream_init", "csvd_stream_push", "csvd_stream_count",
                 "csvd_stream_cluster", "csvd_stream_free",
                 "csvd_cluster", "csvd_tail_grad", "csvd_block_energy", "csvd_set_allocator",
                 "csvd_debug_limits", "csvd_tune_set", "csvd_tune_get", "csvd_tail_energy",
                 "csvd_top_basis", "csvd_randomized_tail", "csvd_score_plan", "csvd_plan_launch",
                 "csvd_plan_status", "csvd_plan_free"):
        getattr(lib, name).restype = C.c_int


def lib_path() -> str:
    return _build.LIB


def lib(require_gpu: bool = True):
    """Load libcsvd.so (built by ``__graft_entry__.build()``)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"csvd CUDA library not built: {path} is missing")
        l = C.CDLL(path)
        _sig(l)
        _LIB = l
    if require_gpu and not torch.cuda.is_available():
        raise RuntimeError("csvd needs a CUDA GPU; none is available")
    return _LIB


def _check(st):
    if st != 0:
        raise CsvdError(st, lib(False).csvd_last_error().decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def block(t: torch.Tensor, m: int = None) -> Block:
    """Descriptor of a row-major (m, k) CUDA tensor (f32 or bf16, unit
    column stride).  The C ABI reads m rows from the pointer, so the row
    count is checked here whenever m is known."""
    if t.dim() != 2:
        raise ValueError("blocks must be 2-D tensors")
    if m is not None and t.shape[0] != m:
        raise ValueError(f"block has {t.shape[0]} rows, expected m = {m}")
    if not t.is_cuda:
        raise ValueError("blocks must be CUDA tensors")
    if t.stride(1) != 1 and t.shape[1] > 1:
        raise ValueError("blocks need unit column stride (row-major)")
    if t.dtype == torch.float32:
        dt = F32
    elif t.dtype == torch.bfloat16:
        dt = BF16
    else:
        raise ValueError("blocks must be float32 or bfloat16")
    ld = t.stride(0) if t.shape[0] > 1 else t.shape[1]
    return Block(t.data_ptr(), t.shape[1], max(ld, t.shape[1]), dt, 0)


def _blocks(ts, m: int = None):
    """Descriptor array; every block must have m rows (default: the first
    block's row count)."""
    if m is None and len(ts) > 0:
        m = ts[0].shape[0]
    arr = (Block * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = block(t, m)
    return arr


class IncrSVD:
    """Rank-r incremental truncated SVD state (Lemma 1, Cor. 3)."""

    def __init__(self, m: int, r: int, precision: str = "plain", stream=None):
        self._lib = lib()
        self.m, self.r = m, r
        self.stream = stream or torch.cuda.current_stream()
        h = C.c_void_p()
        _check(self._lib.csvd_incr_init(C.byref(h), m, r, _prec(precision),
                                        _stream(self.stream)))
        self._h = h
        self._keep = []

    def append(self, A: torch.Tensor):
        b = block(A, self.m)
        _check(self._lib.csvd_incr_append(self._h, C.byref(b)))
        self._keep.append(A)  # borrowed until the stream reaches it
        if len(self._keep) > 64:
            self.stream.synchronize()
            self._keep.clear()
        return self

    def sigma(self) -> np.ndarray:
        out = (C.c_float * self.r)()
        reff = C.c_int32()
        _check(self._lib.csvd_incr_sigma(self._h, out, C.byref(reff)))
        self._keep.clear()
        return np.frombuffer(out, dtype=np.float32, count=reff.value).copy()

    @property
    def rank(self) -> int:
        reff = C.c_int32()
        _check(self._lib.csvd_incr_sigma(self._h, None, C.byref(reff)))
        return reff.value

    def decompose(self, blocks, want_v: bool = True) -> "Decomposition":
        """Final decomposition of the cluster whose blocks were appended:
        U~ = U diag(sigma~) and V_i = A_i^T U diag(sigma~)^-1 from this state."""
        U = self.basis()
        sig = self.sigma()[: U.shape[1]]
        return reconstruct(U, sig, blocks, want_v)

    def basis(self) -> torch.Tensor:
        rk = self.rank
        U = torch.empty(self.m, max(rk, 1), device="cuda", dtype=torch.float32)
        _check(self._lib.csvd_incr_basis(self._h, C.c_void_p(U.data_ptr()), U.stride(0)))
        return U[:, :rk]

    def load(self, U: torch.Tensor, sigma, energy: float, discarded: float):
        """Restore (U, sigma, energy, discarded) -- checkpoint / resume."""
        sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.float32))
        rt = int(sig.size)
        U = U.contiguous() if rt > 0 and U.stride(1) != 1 else U
        ptr = C.c_void_p(U.data_ptr()) if rt > 0 else None
        ld = U.stride(0) if rt > 0 else 1
        _check(self._lib.csvd_incr_load(self._h, ptr, ld, rt,
                                        sig.ctypes.data_as(C.POINTER(C.c_float)),
                                        float(energy), float(discarded)))
        return self

    def tail_error(self) -> dict:
        t, rel, paper, en = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        _check(self._lib.csvd_tail_error(self._h, C.byref(t), C.byref(rel), C.byref(paper),
                                         C.byref(en)))
        self._keep.clear()
        return dict(tail_sq=t.value, tail_rel=rel.value, tail_sq_paper=paper.value,
                    energy=en.value)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.csvd_incr_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _BorrowedState(IncrSVD):
    """A cluster state owned by a Stream (read-only view: sigma, basis,
    tail_error, decompose); released with the stream."""

    def __init__(self, lib_, handle, m, r, stream):
        self._lib, self._h, self.m, self.r, self.stream = lib_, handle, m, r, stream
        self._keep = []

    def append(self, A):
        raise RuntimeError("a stream's cluster states change only through Stream.push")

    def close(self):
        self._h = None


class Stream:
    """Streaming cluster assignment (csvd_stream_*): each pushed block joins
    the accepting cluster with the smallest estimated relative error, or
    starts a new cluster."""

    def __init__(self, m: int, r: int, eps: float, precision: str = "mixed", stream=None):
        self._lib = lib()
        self.m, self.r, self.eps = m, r, float(eps)
        self.stream = stream or torch.cuda.current_stream()
        h = C.c_void_p()
        _check(self._lib.csvd_stream_init(C.byref(h), m, r, self.eps,
                                          _prec(precision),
                                          _stream(self.stream)))
        self._h = h
        self.labels = []

    def push(self, A: torch.Tensor):
        """Returns (cluster index, E~^2 and ||M_C||^2 of that cluster after
        the block joined)."""
        b = block(A, self.m)
        lab, t, en = C.c_int32(), C.c_double(), C.c_double()
        _check(self._lib.csvd_stream_push(self._h, C.byref(b), C.byref(lab), C.byref(t),
                                          C.byref(en)))
        self.labels.append(lab.value)
        return lab.value, t.value, en.value

    @property
    def n_clusters(self) -> int:
        n = C.c_int32()
        _check(self._lib.csvd_stream_count(self._h, C.byref(n)))
        return n.value

    def cluster(self, c: int):
        """(state view, number of blocks) of cluster c."""
        h, nb = C.c_void_p(), C.c_int32()
        _check(self._lib.csvd_stream_cluster(self._h, c, C.byref(h), C.byref(nb)))
        return _BorrowedState(self._lib, h, self.m, self.r, self.stream), nb.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.csvd_stream_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ScoreBatch:
    """Prepared descriptor arrays for repeated ``csvd_score`` calls on the
    same candidates (avoids rebuilding ctypes arrays inside timed loops).

    ``plan()`` goes further (``csvd_score_plan``): the library builds and
    uploads everything once, ``launch()`` then only enqueues the kernels and
    ``check()`` reads the device status; ``graph()`` captures one launch into
    a CUDA graph.  While a plan exists the states must not be appended to and
    the candidate tensors must stay alive (their contents may change)."""

    def __init__(self, states, cand_state, cands, eps, precision="mixed", r_max=None):
        self._lib = lib()
        self.states = states
        self.n = len(cands)
        self.eps = float(eps)
        self.precision = _prec(precision)
        self._st = (C.c_void_p * len(states))(*[s.handle.value for s in states])
        self._cs = (C.c_int32 * self.n)(*[int(x) for x in cand_state])
        self._cb = _blocks(cands, states[0].m)
        self.cands = cands
        self.r_max = r_max or max(s.r for s in states)
        self.sigma = torch.zeros(self.n, self.r_max, device="cuda", dtype=torch.float32)
        self.tail = torch.zeros(self.n, device="cuda", dtype=torch.float64)
        self.paper = torch.zeros(self.n, device="cuda", dtype=torch.float64)
        self.accept = torch.zeros(self.n, device="cuda", dtype=torch.uint8)
        self._plan = None

    def run(self):
        _check(self._lib.csvd_score(self._st, len(self.states), self._cs, self._cb, self.n,
                                    self.eps, self.precision,
                                    C.c_void_p(self.sigma.data_ptr()), self.r_max,
                                    C.c_void_p(self.tail.data_ptr()),
                                    C.c_void_p(self.paper.data_ptr()),
                                    C.c_void_p(self.accept.data_ptr())))
        return self

    def plan(self):
        if self._plan is None:
            h = C.c_void_p()
            _check(self._lib.csvd_score_plan(self._st, len(self.states), self._cs, self._cb,
                                             self.n, self.eps, self.precision,
                                             C.c_void_p(self.sigma.data_ptr()), self.r_max,
                                             C.c_void_p(self.tail.data_ptr()),
                                             C.c_void_p(self.paper.data_ptr()),
                                             C.c_void_p(self.accept.data_ptr()), C.byref(h)))
            self._plan = h
        return self

    def launch(self, stream=None):
        """Enqueue one evaluation of the plan (on ``stream``, else the
        states' stream); no host work, no synchronisation."""
        _check(self._lib.csvd_plan_launch(self.plan()._plan, _stream(stream) if stream else None))
        return self

    def check(self, stream=None):
        """Synchronise and raise for device-side failures since the last check."""
        if self._plan is not None:
            _check(self._lib.csvd_plan_status(self._plan, _stream(stream) if stream else None))
        return self

    def graph(self):
        """One plan launch captured into a ``torch.cuda.CUDAGraph`` (after an
        eager launch that sets the kernels' limits); replaying it writes the
        same outputs."""
        self.launch().check()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=side):
            self.launch(torch.cuda.current_stream())
        return g

    def close(self):
        if self._plan is not None:
            self._lib.csvd_plan_free(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ScoreColumns:
    """Repeated ``csvd_score_columns`` calls: one-column candidates given as
    the rows of ``Xt`` (n x m, f32, CUDA, unit column stride), candidate j
    scored against ``states[cand_state[j]]`` in the mixed form."""

    def __init__(self, states, cand_state, Xt, eps, r_max=None):
        if Xt.dtype != torch.float32 or not Xt.is_cuda or Xt.dim() != 2 or Xt.stride(1) != 1:
            raise ValueError("Xt must be a CUDA float32 matrix with unit column stride")
        if Xt.shape[1] != states[0].m:
            raise ValueError(f"Xt rows have {Xt.shape[1]} entries, expected m = {states[0].m}")
        self._lib = lib()
        self.states = states
        self.Xt = Xt
        self.n = Xt.shape[0]
        self.eps = float(eps)
        self._st = (C.c_void_p * len(states))(*[s.handle.value for s in states])
        self._cs = (C.c_int32 * self.n)(*[int(x) for x in cand_state])
        self.r_max = r_max or max(s.r for s in states)
        self.sigma = torch.zeros(self.n, self.r_max, device="cuda", dtype=torch.float32)
        self.tail = torch.zeros(self.n, device="cuda", dtype=torch.float64)
        self.paper = torch.zeros(self.n, device="cuda", dtype=torch.float64)
        self.accept = torch.zeros(self.n, device="cuda", dtype=torch.uint8)

    def run(self):
        _check(self._lib.csvd_score_columns(self._st, len(self.states), self._cs,
                                            C.c_void_p(self.Xt.data_ptr()), self.Xt.stride(0),
                                            self.n, self.eps, C.c_void_p(self.sigma.data_ptr()),
                                            self.r_max, C.c_void_p(self.tail.data_ptr()),
                                            C.c_void_p(self.paper.data_ptr()),
                                            C.c_void_p(self.accept.data_ptr())))
        return self


def score_columns(states, cand_state, Xt, eps):
    """One-column candidates (rows of ``Xt``); returns (sigma, tail_sq,
    tail_paper, accept) as CUDA tensors."""
    b = ScoreColumns(states, cand_state, Xt, eps).run()
    return b.sigma, b.tail, b.paper, b.accept


def score(states, cand_state, cands, eps, precision="mixed"):
    """Batched merge evaluations; returns (sigma, tail_sq, tail_paper, accept)
    as CUDA tensors."""
    b = ScoreBatch(states, cand_state, cands, eps, precision).run()
    return b.sigma, b.tail, b.paper, b.accept


def score_one_noalloc(state: IncrSVD, A: torch.Tensor, eps: float, sigma=None, tail=None,
                      paper=None, accept=None):
    """Mixed-form merge evaluation of one candidate without any device
    allocation inside the library (scratch is a fixed device array).  The
    output tensors may be passed in; otherwise they are created here by
    torch, before the call."""
    if sigma is None:
        sigma = torch.zeros(state.r, device="cuda", dtype=torch.float32)
    if tail is None:
        tail = torch.zeros(1, device="cuda", dtype=torch.float64)
    if paper is None:
        paper = torch.zeros(1, device="cuda", dtype=torch.float64)
    if accept is None:
        accept = torch.zeros(1, device="cuda", dtype=torch.uint8)
    b = block(A, state.m)
    _check(lib().csvd_score_one_noalloc(state.handle, C.byref(b), float(eps),
                                        C.c_void_p(sigma.data_ptr()), C.c_void_p(tail.data_ptr()),
                                        C.c_void_p(paper.data_ptr()),
                                        C.c_void_p(accept.data_ptr())))
    return sigma, tail, paper, accept


def block_energy(blocks):
    m = blocks[0].shape[0]
    out = (C.c_double * len(blocks))()
    _check(lib().csvd_block_energy(_blocks(blocks), len(blocks), m, _stream(), out))
    return np.frombuffer(out, dtype=np.float64).copy()


def bounds(blocks, r):
    """Weyl (Thm. 1), residual (Cor. 1) and plug-in (Cor. 2) values and the
    energy, for the blocks in the given order."""
    m = blocks[0].shape[0]
    w, res, plug, en = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    _check(lib().csvd_bounds(_blocks(blocks), len(blocks), m, r, _stream(), C.byref(w),
                             C.byref(res), C.byref(plug), C.byref(en)))
    return dict(weyl_sq=w.value, residual_sq=res.value, plugin_sq=plug.value, energy=en.value)


def cluster(blocks, r, eps, algo="approx", sort_mode="frobenius", precision="plain"):
    """Algorithms 1-3 (Appendix E).  Returns labels, clusters (members in
    label order), per-cluster certificate values, energies and the
    compression ratio."""
    n = len(blocks)
    m = blocks[0].shape[0]
    labels = (C.c_int32 * n)()
    est = (C.c_double * n)()
    en = (C.c_double * n)()
    ratio = C.c_double()
    _check(lib().csvd_cluster(_blocks(blocks), n, m, r, float(eps), ALGO[algo], SORT[sort_mode],
                              _prec(precision), _stream(), labels, est,
                              en, C.byref(ratio)))
    lab = list(labels)
    k = max(lab) + 1
    return dict(labels=lab, n_clusters=k, estimate_sq=list(est)[:k], energy=list(en)[:k],
                compression_ratio=ratio.value)


def tail_grad(U: torch.Tensor, blocks, g: float = 1.0):
    """dA_j = 2 g (I - U U^T) A_j for every block (new f32 tensors)."""
    m = blocks[0].shape[0]
    if U.shape[0] != m:
        raise ValueError(f"U has {U.shape[0]} rows, the blocks {m}")
    grads = [torch.empty_like(b, dtype=torch.float32) for b in blocks]
    U = U.contiguous() if U.stride(1) != 1 else U
    _check(lib().csvd_tail_grad(C.c_void_p(U.data_ptr()), U.stride(0), m, U.shape[1],
                                _blocks(blocks), _blocks(grads), len(blocks), float(g),
                                _stream()))
    return grads


class Decomposition:
    """Final decomposition of one cluster: U~ = U diag(s) and the coefficient
    blocks V_i (k_i x r), so that A^_i = U~ V_i^T; per-block residual and
    block energies (FP64) and the cluster's relative reconstruction error."""

    def __init__(self, Ut, V, resid_sq, energy):
        self.Ut, self.V = Ut, V
        self.resid_sq, self.energy = resid_sq, energy

    @property
    def rel_error(self) -> float:
        tot = float(self.energy.sum())
        return math.sqrt(float(self.resid_sq.sum()) / tot) if tot > 0 else 0.0

    @property
    def memory(self) -> int:
        """Stored numbers r (m + N_c)."""
        return self.Ut.shape[0] * self.Ut.shape[1] + sum(v.shape[0] * v.shape[1] for v in self.V)


def reconstruct(U: torch.Tensor, s, blocks, want_v: bool = True) -> Decomposition:
    """Decomposition of a cluster from its basis U (m x r) and singular
    values s (r): V_i = A_i^T U diag(s)^-1, residual energies from the
    explicit residuals A_i - U U^T A_i."""
    m, r = U.shape
    U = U.contiguous().float()
    sd = torch.as_tensor(np.asarray(s, dtype=np.float32), device="cuda").contiguous()
    n = len(blocks)
    V = [torch.empty(b.shape[1], r, device="cuda", dtype=torch.float32) for b in blocks] if want_v else []
    vptr = (C.c_void_p * n)(*[v.data_ptr() for v in V]) if want_v else None
    Ut = torch.empty(m, r, device="cuda", dtype=torch.float32)
    res = (C.c_double * max(n, 1))()
    en = (C.c_double * max(n, 1))()
    _check(lib().csvd_reconstruct(C.c_void_p(U.data_ptr()), U.stride(0), C.c_void_p(sd.data_ptr()), m,
                                  r, _blocks(blocks, m), n, C.c_void_p(Ut.data_ptr()), r, vptr, r,
                                  _stream(), res, en))
    return Decomposition(Ut, V, np.array(res[:n], dtype=np.float64),
                         np.array(en[:n], dtype=np.float64))


def gram_apply(U: torch.Tensor, blocks) -> torch.Tensor:
    """Y = sum_j A_j (A_j^T U) (one subspace-iteration sweep)."""
    m, r = U.shape
    U = U.contiguous()
    Y = torch.empty(m, r, device="cuda", dtype=torch.float32)
    _check(lib().csvd_gram_apply(C.c_void_p(U.data_ptr()), U.stride(0), m, r, _blocks(blocks, m),
                                 len(blocks), C.c_void_p(Y.data_ptr()), Y.stride(0), _stream()))
    return Y


def top_basis(blocks, r, working_rank=None, refine=2):
    """Top-r left basis of the concatenation (csvd_top_basis): incremental
    estimator at ``working_rank``, then ``refine`` subspace-iteration sweeps."""
    m = blocks[0].shape[0]
    U = torch.empty(m, r, device="cuda", dtype=torch.float32)
    reff = C.c_int32()
    _check(lib().csvd_top_basis(_blocks(blocks, m), len(blocks), m, r, int(working_rank or r),
                                int(refine), _stream(), C.c_void_p(U.data_ptr()), U.stride(0),
                                C.byref(reff)))
    return U[:, :reff.value]


def residual_energy(U: torch.Tensor, blocks) -> np.ndarray:
    """||(I - U U^T) A_j||_F^2 of every block (csvd_tail_energy), FP64."""
    m, r = U.shape
    U = U.contiguous()
    out = (C.c_double * max(len(blocks), 1))()
    _check(lib().csvd_tail_energy(C.c_void_p(U.data_ptr()), U.stride(0), m, r, _blocks(blocks, m),
                                  len(blocks), _stream(), out))
    return np.frombuffer(out, dtype=np.float64, count=len(blocks)).copy()


def randomized_tail(blocks, omegas, r, power_iters=1, want_basis=False):
    """Randomized range-finder tail estimate (csvd_randomized_tail): the
    explicit residual energy of the top-r left singular vectors of the
    sketch sum_i A_i Omega_i after ``power_iters`` power iterations.
    ``omegas``: CUDA float32 tensors (k_i x l)."""
    m = blocks[0].shape[0]
    l = int(omegas[0].shape[1])
    om = [o.contiguous() for o in omegas]
    for b, o in zip(blocks, om):
        if o.shape != (b.shape[1], l) or o.dtype != torch.float32 or not o.is_cuda:
            raise ValueError("each Omega_i must be a CUDA float32 (k_i x l) tensor")
    ptrs = (C.c_void_p * len(om))(*[o.data_ptr() for o in om])
    t = C.c_double()
    U = torch.empty(m, r, device="cuda", dtype=torch.float32) if want_basis else None
    _check(lib().csvd_randomized_tail(_blocks(blocks, m), ptrs, len(blocks), m, r, l,
                                      int(power_iters), _stream(), C.byref(t),
                                      C.c_void_p(U.data_ptr()) if U is not None else None,
                                      r))
    return (t.value, U) if want_basis else t.value


class TailEnergy(torch.autograd.Function):
    """E = sum_j ||(I - U_r U_r^T) A_j||_F^2 with U_r the top-r basis from the
    incremental estimator; backward dA_j = 2 (I - U_r U_r^T) A_j * gE
    (the Eckart-Young tail gradient, valid when sigma_r > sigma_{r+1}).  U_r
    is recomputed in the backward instead of being stored."""

    @staticmethod
    def forward(ctx, r, working_rank, *blocks):
        U = top_basis(list(blocks), r, working_rank)
        e = float(residual_energy(U, list(blocks)).sum())
        ctx.r, ctx.working_rank = r, working_rank
        ctx.save_for_backward(*blocks)
        return torch.tensor(e, dtype=torch.float64, device=blocks[0].device)

    @staticmethod
    def backward(ctx, gE):
        blocks = ctx.saved_tensors
        U = top_basis(list(blocks), ctx.r, ctx.working_rank)
        grads = tail_grad(U, list(blocks), float(gE))
        return (None, None, *grads)


def tail_energy(blocks, r, working_rank=None):
    return TailEnergy.apply(r, working_rank, *blocks)


def debug_limits(jacobi_sweeps: int = -1, solver_iters: int = -1, wait_ns: int = -1,
                 stall_gram: bool = False):
    """Failure-path test hook (csvd_debug_limits): solver caps, the
    tensor-core pipeline wait limit and its never-arriving barrier, for the
    current device; -1 / False restore."""
    _check(lib().csvd_debug_limits(jacobi_sweeps, solver_iters, wait_ns, 1 if stall_gram else 0))


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib(False).csvd_launch_count())


def profile(enable: bool):
    _check(lib(False).csvd_profile(1 if enable else 0))


def profile_report() -> dict:
    """{kernel name: (launches, total device ms)} from the CUDA events
    recorded on each launch stream since ``profile(True)``."""
    buf = C.create_string_buffer(1 << 16)
    _check(lib(False).csvd_profile_report(buf, len(buf)))
    out = {}
    for line in buf.value.decode().splitlines():
        name, n, ms = line.split()
        out[name] = (int(n), float(ms))
    return out
