"""Python binding of the GB300 RCB tree library (``include/rcb.h``, ``librcb.so``).

Argument marshalling only: every step of the build, the walk, the neighbour search, gravity
and its gradient runs in the library's CUDA kernels.  Tensors are torch CUDA tensors (device
memory and streams come from PyTorch).  There is no CPU fallback: if ``librcb.so`` is missing
the functions raise.

The function names mirror the C ABI (``rcb_build``, ``rcb_neighbours``, ``rcb_gravity``,
``rcb_gravity_backward``, ``rcb_refit``, ...); ``RCBTree`` wraps a tree handle and
``rcb_gravity_fn`` is the ``torch.autograd.Function`` over gravity.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librcb.so")

RCB_OK, RCB_ERR_ARG, RCB_ERR_ALLOC, RCB_ERR_CAPACITY, RCB_ERR_CUDA, RCB_ERR_LIMIT, RCB_ERR_STATE = 0, -1, -2, -3, -4, -5, -6
RCB_FP64, RCB_MIXED = 0, 1
_PRECISION = {"fp64": RCB_FP64, "mixed": RCB_MIXED, RCB_FP64: RCB_FP64, RCB_MIXED: RCB_MIXED}

RCB_FLAG_TIMING = 1
RCB_FLAG_CENTRE_OF_NUMBER = 2
RCB_FLAG_MAC_ONLY = 4
RCB_FLAG_MEDIAN_SPLIT = 8
_SPLIT_FLAG = {"mass": 0, "number": RCB_FLAG_CENTRE_OF_NUMBER, "median": RCB_FLAG_MEDIAN_SPLIT}
SYMBOLS = ["rcb_build", "rcb_neighbours", "rcb_gravity", "rcb_gravity_neighbours", "rcb_gravity_backward", "rcb_refit", "rcb_update", "rcb_density", "rcb_set_precision",
           "rcb_tree_info", "rcb_export_topology", "rcb_export_lists", "rcb_stage_times", "rcb_free", "rcb_strerror",
           "rcb_neighbour_offsets_noalloc"]
STAGES = ["ingest", "levels", "subtrees", "leaves", "walk", "build", "nb_count", "nb_fill", "nb_sort", "far", "near",
          "backward"]

_lock = threading.Lock()
_lib = None


class RCBError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})")


class rcb_params(ctypes.Structure):
    _fields_ = [("n_ll", ctypes.c_int32), ("precision", ctypes.c_int32), ("theta", ctypes.c_double),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


def build(verbose: bool = False, force: bool = False) -> str:
    from . import _build
    return _build.build(verbose=verbose, force=force)


def lib():
    """The loaded C library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1108_0028_gb300.build()")
            L = ctypes.CDLL(LIB_PATH)
            P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            sig = {
                "rcb_build": (ctypes.c_int, [P, P, P, I64, ctypes.POINTER(rcb_params), P, P, P, P, ctypes.POINTER(P)]),
                "rcb_neighbours": (ctypes.c_int, [P, P, P, I64, ctypes.POINTER(I64), P]),
                "rcb_gravity": (ctypes.c_int, [P, P, P, P]),
                "rcb_gravity_neighbours": (ctypes.c_int, [P, P, P, P, ctypes.POINTER(I64), P]),
                "rcb_gravity_backward": (ctypes.c_int, [P, P, P, P, P, P]),
                "rcb_refit": (ctypes.c_int, [P, P, P, P]),
                "rcb_update": (ctypes.c_int, [P, P, P, P, P, P]),
                "rcb_density": (ctypes.c_int, [P, P, P, P, P]),
                "rcb_set_precision": (ctypes.c_int, [P, I32]),
                "rcb_tree_info": (ctypes.c_int, [P, P]),
                "rcb_export_topology": (ctypes.c_int, [P] + [P] * 16 + [P]),
                "rcb_export_lists": (ctypes.c_int, [P, P, P, P, I64, P, P, I64, P]),
                "rcb_stage_times": (ctypes.c_int, [P, P, P]),
                "rcb_neighbour_offsets_noalloc": (ctypes.c_int, [P, P, ctypes.POINTER(I64), P]),
                "rcb_free": (None, [P]),
                "rcb_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().rcb_strerror(int(status)).decode()


def _check(status: int, what: str) -> None:
    if status != RCB_OK:
        raise RCBError(status, what)


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _cuda_f64(t, shape, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64 or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 tensor of shape {tuple(shape)}")
    return t


# ---------------------------------------------------------------------------------------------
# C-ABI mirrors (argument marshalling only)

# torch's caching allocator behind the library's allocator callbacks (rcb_alloc_fn, rcb_free_fn):
# the tree's device arrays then come from, and return to, the same pool as PyTorch's tensors
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


def _torch_alloc(nbytes, ctx, stream):
    try:
        return _torch().cuda.caching_allocator_alloc(int(nbytes), None, int(stream or 0))
    except Exception:  # the library reports RCB_ERR_ALLOC
        return None


def _torch_free(ptr, ctx, stream):
    try:
        if ptr:
            _torch().cuda.caching_allocator_delete(int(ptr))
    except Exception:  # torch already torn down at interpreter exit
        pass


_TORCH_ALLOC = _ALLOC_FN(_torch_alloc)
_TORCH_FREE = _FREE_FN(_torch_free)


def rcb_build(x, m, h, n_ll=12, theta=0.7, precision="mixed", tree=None, stream=None, flags=0,
              allocator: str = "torch"):
    """Build (or rebuild in place) a tree; returns the handle (ctypes.c_void_p).  allocator:
    "torch" (the caching allocator, through rcb_alloc_fn / rcb_free_fn) or "cuda" (the library's
    own cudaMallocAsync / cudaFreeAsync).  A rebuild keeps the tree's first allocator."""
    N = x.shape[0] if x.dim() == 2 else 0
    _cuda_f64(x, (N, 3), "x")
    _cuda_f64(m, (N,), "m")
    _cuda_f64(h, (N,), "h")
    if allocator not in ("torch", "cuda"):
        raise ValueError("allocator must be 'torch' or 'cuda'")
    p = rcb_params(int(n_ll), _PRECISION[precision], float(theta), int(flags), 0)
    handle = tree if tree is not None else ctypes.c_void_p(None)
    fa, ff = (_TORCH_ALLOC, _TORCH_FREE) if allocator == "torch" else (None, None)
    st = lib().rcb_build(_dptr(x), _dptr(m), _dptr(h), N, ctypes.byref(p), fa, ff, None, _stream_ptr(stream),
                         ctypes.byref(handle))
    _check(st, "rcb_build")
    return handle


def rcb_neighbours(tree, offsets, idx, capacity, stream=None):
    needed = ctypes.c_int64(0)
    st = lib().rcb_neighbours(tree, _dptr(offsets), _dptr(idx), int(capacity), ctypes.byref(needed),
                              _stream_ptr(stream))
    return st, needed.value


def rcb_gravity(tree, acc, pot=None, stream=None):
    _check(lib().rcb_gravity(tree, _dptr(acc), _dptr(pot), _stream_ptr(stream)), "rcb_gravity")


def rcb_gravity_neighbours(tree, acc, pot, offsets, stream=None):
    needed = ctypes.c_int64(0)
    _check(lib().rcb_gravity_neighbours(tree, _dptr(acc), _dptr(pot), _dptr(offsets), ctypes.byref(needed),
                                        _stream_ptr(stream)), "rcb_gravity_neighbours")
    return needed.value


def rcb_gravity_backward(tree, g_acc, g_pot, g_x, g_m, stream=None):
    _check(lib().rcb_gravity_backward(tree, _dptr(g_acc), _dptr(g_pot), _dptr(g_x), _dptr(g_m), _stream_ptr(stream)),
           "rcb_gravity_backward")


def rcb_refit(tree, x, m, stream=None):
    _check(lib().rcb_refit(tree, _dptr(x), _dptr(m), _stream_ptr(stream)), "rcb_refit")


def rcb_density(tree, offsets, idx, rho, stream=None) -> None:
    _check(lib().rcb_density(tree, _dptr(offsets), _dptr(idx), _dptr(rho), _stream_ptr(stream)), "rcb_density")


def rcb_update(tree, x, m, h, stream=None) -> bool:
    """Sec. 2.1.8 update: refit and walk again when every particle is still in its ll-cell,
    rebuild otherwise.  Returns True when the tree was rebuilt."""
    flag = np.zeros(1, np.int32)
    _check(lib().rcb_update(tree, _dptr(x), _dptr(m), _dptr(h), _hptr(flag), _stream_ptr(stream)), "rcb_update")
    return bool(flag[0])


def rcb_set_precision(tree, precision):
    _check(lib().rcb_set_precision(tree, _PRECISION[precision]), "rcb_set_precision")


def rcb_tree_info(tree) -> dict:
    info = np.zeros(16, np.int64)
    _check(lib().rcb_tree_info(tree, _hptr(info)), "rcb_tree_info")
    keys = ["N", "L", "nn", "nleaves", "nsinks", "cap_near", "cap_far", "near_total", "far_total", "reach_total",
            "walk_fp64_decisions", "smem_subtrees", "precision", "near_pairs", "candidate_pairs", "launches"]
    return {k: int(info[i]) for i, k in enumerate(keys)}


def rcb_stage_times(tree, stream=None) -> dict:
    ms = np.zeros(16)
    _check(lib().rcb_stage_times(tree, _hptr(ms), _stream_ptr(stream)), "rcb_stage_times")
    return {k: float(ms[i]) for i, k in enumerate(STAGES)}


def rcb_free(tree) -> None:
    if tree is not None and tree.value:
        lib().rcb_free(tree)


# ---------------------------------------------------------------------------------------------
class RCBTree:
    """An RCB tree over CUDA tensors x[N,3], m[N], h[N] (float64)."""

    def __init__(self, x, m, h, n_ll: int = 12, theta: float = 0.7, precision="mixed", stream=None,
                 timing: bool = False, split: str = "mass", mac_only: bool = False):
        """split: "mass" cuts every cell through its centre of mass (Sec. 2.1.3), "number" through
        its centre of number (unit weights; node moments stay mass-weighted), "median" at the
        median position along the longest side (the MPS variant: daughters of floor(n/2) and
        ceil(n/2) particles).  mac_only: near lists from the MAC alone (Sec. 2.5 variant),
        neighbour candidates from a walk of their own."""
        if split not in _SPLIT_FLAG:
            raise ValueError(f"split must be 'mass', 'number' or 'median', not {split!r}")
        self._h = None
        self.n_ll, self.theta, self.precision = n_ll, theta, precision
        self.flags = (RCB_FLAG_TIMING if timing else 0) | _SPLIT_FLAG[split] | (RCB_FLAG_MAC_ONLY if mac_only else 0)
        self._h = rcb_build(x, m, h, n_ll, theta, precision, None, stream, self.flags)
        self.N = x.shape[0]
        self.device = x.device
        self._nb_cap = 0

    def rebuild(self, x, m, h, stream=None):
        self._h = rcb_build(x, m, h, self.n_ll, self.theta, self.precision, self._h, stream, self.flags)
        self.N = x.shape[0]

    def stage_times(self, stream=None) -> dict:
        return rcb_stage_times(self._h, stream)

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        return rcb_tree_info(self._h)

    def set_precision(self, precision) -> None:
        rcb_set_precision(self._h, precision)
        self.precision = precision

    def neighbours(self, stream=None, capacity_hint: int | None = None):
        """CSR neighbour lists (offsets int64[N+1], idx int32[total]) in original order."""
        torch = _torch()
        offsets = torch.empty(self.N + 1, dtype=torch.int64, device=self.device)
        cap = capacity_hint if capacity_hint is not None else max(self._nb_cap, 1)
        idx = torch.empty(cap, dtype=torch.int32, device=self.device)
        st, needed = rcb_neighbours(self._h, offsets, idx, cap, stream)
        if st == RCB_ERR_CAPACITY:
            idx = torch.empty(max(needed, 1), dtype=torch.int32, device=self.device)
            st, needed = rcb_neighbours(self._h, offsets, idx, idx.numel(), stream)
        _check(st, "rcb_neighbours")
        self._nb_cap = max(self._nb_cap, needed)
        return offsets, idx[:needed]

    def gravity(self, stream=None, with_pot: bool = True):
        torch = _torch()
        acc = torch.empty((self.N, 3), dtype=torch.float64, device=self.device)
        pot = torch.empty(self.N, dtype=torch.float64, device=self.device) if with_pot else None
        rcb_gravity(self._h, acc, pot, stream)
        return acc, pot

    def gravity_neighbours(self, stream=None, with_pot: bool = True):
        """Forces and neighbour lists from one pass over the near lists: (acc, pot, offsets, idx)."""
        torch = _torch()
        acc = torch.empty((self.N, 3), dtype=torch.float64, device=self.device)
        pot = torch.empty(self.N, dtype=torch.float64, device=self.device) if with_pot else None
        offsets = torch.empty(self.N + 1, dtype=torch.int64, device=self.device)
        needed = rcb_gravity_neighbours(self._h, acc, pot, offsets, stream)
        idx = torch.empty(max(needed, 1), dtype=torch.int32, device=self.device)
        st, needed = rcb_neighbours(self._h, offsets, idx, idx.numel(), stream)
        _check(st, "rcb_neighbours")
        self._nb_cap = max(self._nb_cap, needed)
        return acc, pot, offsets, idx[:needed]

    def gravity_backward(self, g_acc, g_pot=None, stream=None):
        torch = _torch()
        g_acc = g_acc.contiguous()
        g_pot = None if g_pot is None else g_pot.contiguous()
        gx = torch.empty((self.N, 3), dtype=torch.float64, device=self.device)
        gm = torch.empty(self.N, dtype=torch.float64, device=self.device)
        rcb_gravity_backward(self._h, g_acc, g_pot, gx, gm, stream)
        return gx, gm

    def refit(self, x, m, stream=None):
        rcb_refit(self._h, x, m, stream)

    def density(self, offsets, idx, stream=None):
        """SPH density (float64, original order) over the CSR of neighbours()."""
        torch = _torch()
        rho = torch.empty(self.N, dtype=torch.float64, device=self.device)
        rcb_density(self._h, offsets, idx, rho, stream)
        return rho

    def update(self, x, m, h, stream=None) -> bool:
        """Integrity check, then refit + walk or rebuild (Sec. 2.1.8); True when rebuilt."""
        return rcb_update(self._h, x, m, h, stream)

    def export_topology(self, stream=None) -> dict:
        inf = self.info()
        N, nn = inf["N"], inf["nn"]
        out = {"leaf_of": np.zeros(N, np.int32), "perm": np.zeros(N, np.int32), "first": np.zeros(nn, np.int64),
               "count": np.zeros(nn, np.int64), "axis": np.zeros(nn, np.int32), "split": np.zeros(nn),
               "sums": np.zeros((nn, 4, 2), np.int64), "mass": np.zeros(nn), "com": np.zeros((nn, 3)),
               "bmin": np.zeros((nn, 3)), "bmax": np.zeros((nn, 3)), "rg": np.zeros((nn, 3)), "H": np.zeros(nn),
               "hint": np.zeros(nn), "hnode": np.zeros(nn), "Q": np.zeros((nn, 6))}
        keys = ["leaf_of", "perm", "first", "count", "axis", "split", "sums", "mass", "com", "bmin", "bmax", "rg", "H",
                "hint", "hnode", "Q"]
        _check(lib().rcb_export_topology(self._h, *[_hptr(out[k]) for k in keys], _stream_ptr(stream)),
               "rcb_export_topology")
        return out

    def export_lists(self, stream=None) -> dict:
        inf = self.info()
        nl = inf["nleaves"]
        near_off = np.zeros(nl + 1, np.int64)
        far_off = np.zeros(nl + 1, np.int64)
        near_ids = np.zeros(max(inf["near_total"], 1), np.int32)
        near_reach = np.zeros(max(inf["near_total"], 1), np.uint8)
        far_ids = np.zeros(max(inf["far_total"], 1), np.int32)
        _check(lib().rcb_export_lists(self._h, _hptr(near_off), _hptr(near_ids), _hptr(near_reach), near_ids.size,
                                      _hptr(far_off), _hptr(far_ids), far_ids.size, _stream_ptr(stream)),
               "rcb_export_lists")
        return {"near_off": near_off, "near_ids": near_ids[:inf["near_total"]],
                "near_reach": near_reach[:inf["near_total"]], "far_off": far_off,
                "far_ids": far_ids[:inf["far_total"]]}

    def free(self):
        if self._h is not None:
            rcb_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _make_gravity_fn():
    torch = _torch()

    class _RCBGravity(torch.autograd.Function):
        """Gravity (acc, pot) of particles x, m with constant h; backward through the frozen tree."""

        @staticmethod
        def forward(ctx, x, m, h, n_ll, theta, precision):
            tree = RCBTree(x.detach().contiguous(), m.detach().contiguous(), h.detach().contiguous(), n_ll, theta,
                           precision)
            acc, pot = tree.gravity()
            ctx.tree = tree
            return acc, pot

        @staticmethod
        def backward(ctx, g_acc, g_pot):
            torch_ = _torch()
            if g_acc is None:
                g_acc = torch_.zeros((ctx.tree.N, 3), dtype=torch_.float64, device=ctx.tree.device)
            gx, gm = ctx.tree.gravity_backward(g_acc, g_pot)
            return gx, gm, None, None, None, None

    return _RCBGravity


_gravity_fn = None


def rcb_gravity_fn(x, m, h, n_ll: int = 12, theta: float = 0.7, precision="mixed"):
    """Differentiable gravity: returns (acc[N,3], pot[N]); gradients flow to x and m."""
    global _gravity_fn
    if _gravity_fn is None:
        _gravity_fn = _make_gravity_fn()
    return _gravity_fn.apply(x, m, h, n_ll, theta, precision)


def alu_rates(sms: int, iters: int = 4096) -> dict:
    """Measured arithmetic rates of the current GPU from the probe library ``libpeak.so``
    (``peak/alu_rate.cu``): FP32 FMA, paired FP32 FMA, MUFU reciprocal square root (tera-operations
    per second, FMA = 2 flops) and FP64 FMA.  Best of three runs of each probe on ``sms`` x 4
    blocks of 256 threads.  A diagnostic of the benchmark; it changes no device setting."""
    import torch

    path = os.path.join(_HERE, "libpeak.so")
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1108_0028_gb300.build()")
    L = ctypes.CDLL(path)
    L.alu_rate_run.restype = ctypes.c_double
    L.alu_rate_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                               ctypes.POINTER(ctypes.c_double)]
    blocks, threads = 4 * sms, 256
    out = torch.empty(blocks * threads, dtype=torch.float32, device="cuda")
    res = {}
    for which, name, it in ((0, "ffma_tflops", iters), (1, "ffma2_tflops", iters), (2, "rsqrt_tops", iters // 4),
                            (3, "dfma_tflops", max(1, iters // 64))):
        best = 0.0
        for _ in range(4):   # the first run is a warm-up
            ops = ctypes.c_double(0.0)
            ms = L.alu_rate_run(which, blocks, threads, it, ctypes.c_void_p(out.data_ptr()), ctypes.byref(ops))
            if ms <= 0:
                raise RuntimeError("ALU rate probe failed")
            best = max(best, ops.value / (ms * 1e-3) / 1e12)
        res[name] = round(best, 3)
    return res
