"""ctypes wrapper of the FP64 CPU oracle (``rcb_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` are the only code that may import this package.  The CUDA library and its
Python binding never import it, and it imports nothing from them.

The C source is compiled on first use (or by ``build()``) into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rcb_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_ALLOC, ERR_CAPACITY, ERR_STATE = 0, -1, -2, -3, -4


def build(force: bool = False) -> str:
    """Compile the oracle (plain C11, FP64, no FMA contraction, OpenMP over sinks)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
            "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            sig = {
                "orc_depth": (ctypes.c_int, [_I64, ctypes.c_int32]),
                "orc_build": (_P, [_P, _P, _P, _I64, ctypes.c_int32, _P]),
                "orc_build_split": (_P, [_P, _P, _P, _I64, ctypes.c_int32, ctypes.c_int, _P]),
                "orc_free": (None, [_P]),
                "orc_info": (None, [_P, _P]),
                "orc_export_nodes": (None, [_P] + [_P] * 14),
                "orc_export_perm": (None, [_P, _P]),
                "orc_export_fixed": (None, [_P, _P]),
                "orc_i128_to_double": (_D, [_I64, _I64]),
                "orc_walk": (ctypes.c_int, [_P, _D, _P, _I64]),
                "orc_list_sizes": (None, [_P, _P]),
                "orc_export_lists": (None, [_P, _P, _P, _P, _P, _P]),
                "orc_neighbours": (_I64, [_P, _P, _P, _I64]),
                "orc_brute_neighbours": (_I64, [_P, _P, _I64, _P, _P, _I64]),
                "orc_kernel_S": (_D, [_D, _D]),
                "orc_kernel_S_over_r": (_D, [_D, _D]),
                "orc_kernel_dSr_over_r": (_D, [_D, _D]),
                "orc_kernel_phi": (_D, [_D, _D]),
                "orc_dinv_r": (_D, [ctypes.c_int, _P, _P]),
                "orc_far_coeffs": (None, [_P, _D, _P, _P]),
                "orc_taylor_eval": (None, [_P, _P, _P, _P]),
                "orc_gravity": (ctypes.c_int, [_P, _P, _P]),
                "orc_direct": (None, [_P, _P, _P, _I64, _P, _I64, _P, _P]),
                "orc_direct_grad": (None, [_P, _P, _P, _I64, _P, _P, _P, _P]),
                "orc_refit": (ctypes.c_int, [_P, _P, _P]),
                "orc_update": (ctypes.c_int, [_P, _P, _P, _P, _P]),
                "orc_walk_mac_only": (ctypes.c_int, [_P, ctypes.c_double]),
                "orc_walk_bisection_box": (ctypes.c_int, [_P, ctypes.c_double]),
                "orc_kernel_W": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
                "orc_density_csr": (ctypes.c_int, [ctypes.c_int64, _P, _P, _P, _P, _P, _P]),
                "orc_gravity_backward": (ctypes.c_int, [_P, _P, _P, _P, _P]),
                "orc_num_threads": (ctypes.c_int, []),
                "orc_set_num_threads": (None, [ctypes.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def depth(N: int, n_ll: int = 12) -> int:
    return lib().orc_depth(int(N), int(n_ll))


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


def i128_to_double(v: int) -> float:
    lo = v & ((1 << 64) - 1)
    hi = v >> 64
    if lo >= 1 << 63:
        lo -= 1 << 64
    return lib().orc_i128_to_double(lo, hi)


def kernel_S(r, h):
    return lib().orc_kernel_S(float(r), float(h))


def kernel_S_over_r(r, h):
    return lib().orc_kernel_S_over_r(float(r), float(h))


def kernel_dSr_over_r(r, h):
    return lib().orc_kernel_dSr_over_r(float(r), float(h))


def kernel_phi(r, h):
    return lib().orc_kernel_phi(float(r), float(h))


def dinv_r(idx, x) -> float:
    idx_a = np.ascontiguousarray(list(idx) + [0] * (8 - len(idx)), dtype=np.int32)
    x_a = _f64(x)
    return lib().orc_dinv_r(len(idx), _ptr(idx_a), _ptr(x_a))


def far_coeffs(R, M, q6) -> np.ndarray:
    C = np.zeros(20)
    R_a, q_a = _f64(R), _f64(q6)
    lib().orc_far_coeffs(_ptr(R_a), float(M), _ptr(q_a), _ptr(C))
    return C


def taylor_eval(C, d):
    C_a, d_a = _f64(C), _f64(d)
    phi = np.zeros(1)
    acc = np.zeros(3)
    lib().orc_taylor_eval(_ptr(C_a), _ptr(d_a), _ptr(phi), _ptr(acc))
    return float(phi[0]), acc


def kernel_W(r, h):
    return lib().orc_kernel_W(float(r), float(h))


def density(x, m, h, offsets, idx):
    """SPH density by summation over neighbour rows (CSR, original order), FP64."""
    x, m, h = _f64(x, (-1, 3)), _f64(m), _f64(h)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    ix = np.ascontiguousarray(idx, dtype=np.int32)
    rho = np.zeros(x.shape[0])
    r = lib().orc_density_csr(x.shape[0], _ptr(x), _ptr(m), _ptr(h), _ptr(off), _ptr(ix), _ptr(rho))
    if r != OK:
        raise RuntimeError(f"oracle density failed: {r}")
    return rho


def direct(x, m, h, targets=None):
    """Direct kernel-softened sum (acc[nt,3], pot[nt]) for the given original indices."""
    x, m, h = _f64(x, (-1, 3)), _f64(m), _f64(h)
    N = x.shape[0]
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = N if t is None else t.shape[0]
    acc = np.zeros((nt, 3))
    pot = np.zeros(nt)
    lib().orc_direct(_ptr(x), _ptr(m), _ptr(h), N, _ptr(t), nt, _ptr(acc), _ptr(pot))
    return acc, pot


def direct_grad(x, m, h, gacc, gpot=None):
    x, m, h = _f64(x, (-1, 3)), _f64(m), _f64(h)
    N = x.shape[0]
    ga = _f64(gacc, (-1, 3))
    gp = None if gpot is None else _f64(gpot)
    gx = np.zeros((N, 3))
    gm = np.zeros(N)
    lib().orc_direct_grad(_ptr(x), _ptr(m), _ptr(h), N, _ptr(ga), _ptr(gp), _ptr(gx), _ptr(gm))
    return gx, gm


def brute_neighbours(x, h):
    x, h = _f64(x, (-1, 3)), _f64(h)
    N = x.shape[0]
    off = np.zeros(N + 1, dtype=np.int64)
    total = lib().orc_brute_neighbours(_ptr(x), _ptr(h), N, _ptr(off), None, 0)
    idx = np.zeros(max(total, 1), dtype=np.int32)
    r = lib().orc_brute_neighbours(_ptr(x), _ptr(h), N, _ptr(off), _ptr(idx), idx.shape[0])
    if r < 0:
        raise RuntimeError(f"oracle brute neighbours failed: {r}")
    return off, idx[:total]


class OracleTree:
    """The oracle's RCB tree (Sec. 2.1) with walk, neighbours, gravity and gradients."""

    def __init__(self, x, m, h, n_ll: int = 12, split: str = "mass"):
        """split: "mass" cuts every cell through its centre of mass (CMS, Sec. 2.1.3), "median"
        through the median position along the longest side (the MPS variant of the same
        section)."""
        if split not in ("mass", "median"):
            raise ValueError("split must be 'mass' or 'median'")
        self.x = _f64(x, (-1, 3))
        self.m = _f64(m)
        self.h = _f64(h)
        self.N = self.x.shape[0]
        st = ctypes.c_int(0)
        self._t = lib().orc_build_split(_ptr(self.x), _ptr(self.m), _ptr(self.h), self.N, int(n_ll),
                                        1 if split == "median" else 0, ctypes.byref(st))
        if not self._t:
            raise ValueError(f"oracle build failed with status {st.value}")
        info = np.zeros(8, dtype=np.int64)
        lib().orc_info(self._t, _ptr(info))
        self.L = int(info[1])
        self.nn = int(info[2])
        self.E = [int(v) for v in info[3:6]]
        self.Em = int(info[6])
        self.n_ll = int(info[7])
        self.walked = False

    def __del__(self):
        t = getattr(self, "_t", None)
        if t:
            lib().orc_free(t)
            self._t = None

    @property
    def nleaves(self) -> int:
        return 1 << self.L

    def nodes(self) -> dict:
        nn = self.nn
        out = {
            "first": np.zeros(nn, np.int64), "count": np.zeros(nn, np.int64),
            "axis": np.zeros(nn, np.int32), "split": np.zeros(nn),
            "sums": np.zeros((nn, 4, 2), np.int64), "mass": np.zeros(nn),
            "com": np.zeros((nn, 3)), "bmin": np.zeros((nn, 3)), "bmax": np.zeros((nn, 3)),
            "rg": np.zeros((nn, 3)), "H": np.zeros(nn), "hint": np.zeros(nn),
            "hnode": np.zeros(nn), "Q": np.zeros((nn, 6)),
        }
        k = ["first", "count", "axis", "split", "sums", "mass", "com", "bmin", "bmax", "rg", "H", "hint", "hnode", "Q"]
        lib().orc_export_nodes(self._t, *[_ptr(out[n]) for n in k])
        return out

    def perm(self) -> np.ndarray:
        p = np.zeros(self.N, np.int32)
        lib().orc_export_perm(self._t, _ptr(p))
        return p

    def fixed(self) -> np.ndarray:
        """Per-particle fixed-point integers [N, 4] (m, m x, m y, m z) in original order."""
        P = np.zeros((self.N, 4), np.int64)
        lib().orc_export_fixed(self._t, _ptr(P))
        return P

    def leaf_of(self) -> np.ndarray:
        """Leaf number (0 .. 2^L - 1) of every particle, in original order."""
        nd = self.nodes()
        perm = self.perm()
        out = np.empty(self.N, np.int64)
        leaf0 = 1 << self.L
        for j in range(self.nleaves):
            f, c = nd["first"][leaf0 + j], nd["count"][leaf0 + j]
            out[perm[f:f + c]] = j
        return out

    def walk(self, theta: float, sinks=None, mac_only: bool = False, mac_box: str = "tight") -> None:
        """mac_only: near lists from the MAC alone (Sec. 2.5 variant); every sink is walked and the
        lists hold no neighbour candidates.  mac_box="bisection": Eq. 4's cell size taken from each
        cell's bisection box instead of the tight box of its particles (the other reading of the
        cell size, for comparison; every sink is walked)."""
        if mac_box == "bisection":
            if sinks is not None or mac_only:
                raise ValueError("the bisection-box walk covers every sink with the default rules")
            r = lib().orc_walk_bisection_box(self._t, float(theta))
            if r != OK:
                raise RuntimeError(f"oracle walk failed: {r}")
            self.walked = True
            return
        if mac_box != "tight":
            raise ValueError(f"unknown mac_box {mac_box!r}")
        if mac_only:
            if sinks is not None:
                raise ValueError("the MAC-only walk covers every sink")
            r = lib().orc_walk_mac_only(self._t, float(theta))
            if r != OK:
                raise RuntimeError(f"oracle walk failed: {r}")
            self.walked = True
            return
        s = None if sinks is None else np.ascontiguousarray(sinks, dtype=np.int32)
        r = lib().orc_walk(self._t, float(theta), _ptr(s), -1 if s is None else s.shape[0])
        if r != OK:
            raise RuntimeError(f"oracle walk failed: {r}")
        self.walked = True

    def lists(self) -> dict:
        sz = np.zeros(3, np.int64)
        lib().orc_list_sizes(self._t, _ptr(sz))
        nl = self.nleaves
        near_off = np.zeros(nl + 1, np.int64)
        far_off = np.zeros(nl + 1, np.int64)
        near_ids = np.zeros(max(sz[0], 1), np.int32)
        near_reach = np.zeros(max(sz[0], 1), np.uint8)
        far_ids = np.zeros(max(sz[1], 1), np.int32)
        lib().orc_export_lists(self._t, _ptr(near_off), _ptr(near_ids), _ptr(near_reach), _ptr(far_off), _ptr(far_ids))
        return {"near_off": near_off, "near_ids": near_ids[:sz[0]], "near_reach": near_reach[:sz[0]],
                "far_off": far_off, "far_ids": far_ids[:sz[1]]}

    def neighbours(self):
        off = np.zeros(self.N + 1, np.int64)
        total = lib().orc_neighbours(self._t, _ptr(off), None, 0)
        if total < 0:
            raise RuntimeError(f"oracle neighbours failed: {total}")
        idx = np.zeros(max(total, 1), np.int32)
        r = lib().orc_neighbours(self._t, _ptr(off), _ptr(idx), idx.shape[0])
        if r < 0:
            raise RuntimeError(f"oracle neighbours failed: {r}")
        return off, idx[:total]

    def gravity(self):
        acc = np.full((self.N, 3), np.nan)
        pot = np.full(self.N, np.nan)
        r = lib().orc_gravity(self._t, _ptr(acc), _ptr(pot))
        if r != OK:
            raise RuntimeError(f"oracle gravity failed: {r}")
        return acc, pot

    def refit(self, x, m) -> None:
        x, m = _f64(x, (-1, 3)), _f64(m)
        r = lib().orc_refit(self._t, _ptr(x), _ptr(m))
        if r != OK:
            raise RuntimeError(f"oracle refit failed: {r}")

    def update(self, x, m, h) -> int:
        """Sec. 2.1.8 tree update: the number of particles that left their ll-cells at positions
        x (original order).  When it is zero, h is replaced, the tree refitted and the lists
        dropped (walk again); otherwise the tree is unchanged (build a new one)."""
        x, m, h = _f64(x, (-1, 3)), _f64(m), _f64(h)
        out = np.zeros(1, np.int64)
        r = lib().orc_update(self._t, _ptr(x), _ptr(m), _ptr(h), _ptr(out))
        if r != OK:
            raise RuntimeError(f"oracle update failed: {r}")
        if out[0] == 0:
            self.x, self.m, self.h = x, m, h
            self.walked = False
        return int(out[0])

    def gravity_backward(self, gacc, gpot=None):
        ga = _f64(gacc, (-1, 3))
        gp = None if gpot is None else _f64(gpot)
        gx = np.zeros((self.N, 3))
        gm = np.zeros(self.N)
        r = lib().orc_gravity_backward(self._t, _ptr(ga), _ptr(gp), _ptr(gx), _ptr(gm))
        if r != OK:
            raise RuntimeError(f"oracle backward failed: {r}")
        return gx, gm
