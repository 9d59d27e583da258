"""CPU timing baseline: the paper's fast transforms on the host cores (Alg. 3 for zeta,
Alg. 4 in the antichain order of Alg. 5 for Moebius), C with OpenMP in mzcpu.c.

It is a reference point for the GPU numbers, not part of the library and not the
parity oracle. Its inputs are a built plan's exported host structures (chains, heights,
the dense niv map), so it times the transforms only, as the paper does. Built with gcc
on first use into cpubase/_build/.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mzcpu.c")
LIB = os.path.join(HERE, "_build", "libmzcpu.so")
_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O3", "-fPIC", "-shared", SRC, "-o", tmp]
    r = subprocess.run(base[:2] + ["-fopenmp"] + base[2:], capture_output=True, text=True)
    if r.returncode != 0:   # no OpenMP: one thread
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"building {SRC} failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.mzcpu_threads.restype = ctypes.c_int
        lib.mzcpu_set_threads.argtypes = [ctypes.c_int]
        for suf in ("f64", "i64"):
            getattr(lib, f"mzcpu_zeta_{suf}").argtypes = [i64, i32, vp, vp, vp, vp, vp, vp]
            getattr(lib, f"mzcpu_mobius_{suf}").argtypes = [i64, i32, vp, vp, vp, vp, i32, vp, vp, vp, vp]
            getattr(lib, f"mzcpu_mobius_u_{suf}").argtypes = [i64, i64, i32, vp, vp, vp, vp, i32, vp, vp, vp, vp]
        _lib = lib
    return _lib


def threads() -> int:
    return _load().mzcpu_threads()


def set_threads(t: int) -> None:
    _load().mzcpu_set_threads(int(t))


class CpuPlan:
    """Host arrays of the paper's method for one poset, from a plan's exports (dense niv map)."""

    def __init__(self, plan, export_niv, export_chain_id, export_chain_pos, export_level, export_ulevel=None):
        info = plan.info
        self.n, self.k = int(info["n"]), int(info["k"])
        n, k = self.n, self.k
        chain = plan.export(export_chain_id).astype(np.int64)
        pos = plan.export(export_chain_pos).astype(np.int64)
        level = plan.export(export_level).astype(np.int64)
        niv = plan.export(export_niv).reshape(n, k)
        lens = np.bincount(chain, minlength=k)
        base = np.concatenate([[0], np.cumsum(lens + 1)])[:k]
        self.S = int(n + k)
        self.chain_base = np.ascontiguousarray(np.concatenate([base, [self.S]]).astype(np.int64))
        self.node_slot = np.ascontiguousarray((base[chain] + 1 + pos).astype(np.int32))
        self.slot_node = np.full(self.S, -1, np.int32)
        self.slot_node[self.node_slot] = np.arange(n, dtype=np.int32)
        self.chain_of = np.ascontiguousarray(chain.astype(np.int32))
        self.N = np.ascontiguousarray(np.where(niv >= 0, self.node_slot[np.maximum(niv, 0)], base[None, :]).astype(np.int32))
        order = np.argsort(level, kind="stable")
        self.lvl_nodes = np.ascontiguousarray(order.astype(np.int32))
        counts = np.bincount(level)[1:]
        self.nlevels = int(counts.size)
        self.lvl_ptr = np.ascontiguousarray(np.concatenate([[0], np.cumsum(counts)]).astype(np.int64))
        self.u_nodes = self.u_ptr = None
        if export_ulevel is not None:   # levels of U's dependency graph, from 0
            ul = plan.export(export_ulevel).astype(np.int64)
            self.u_nodes = np.ascontiguousarray(np.argsort(ul, kind="stable").astype(np.int32))
            uc = np.bincount(ul)
            self.n_ulevels = int(uc.size)
            self.u_ptr = np.ascontiguousarray(np.concatenate([[0], np.cumsum(uc)]).astype(np.int64))
        self.P = None

    def _ptr(self, a):
        return a.ctypes.data

    def _prep(self, x):
        x = np.ascontiguousarray(x)
        if x.dtype == np.float64:
            return x, "f64", np.float64
        return np.ascontiguousarray(x.astype(np.int64)), "i64", np.int64

    def zeta(self, f):
        f, suf, dt = self._prep(f)
        g = np.empty(self.n, dt)
        P = np.empty(self.S, dt)
        getattr(_load(), f"mzcpu_zeta_{suf}")(self.n, self.k, self._ptr(self.chain_base), self._ptr(self.slot_node),
                                               self._ptr(self.N), self._ptr(f), self._ptr(g), self._ptr(P))
        return g

    def mobius_u(self, g):
        """Moebius with U's dependency levels as the schedule (needs export_ulevel)."""
        g, suf, dt = self._prep(g)
        f = np.empty(self.n, dt)
        P = np.empty(self.S, dt)
        getattr(_load(), f"mzcpu_mobius_u_{suf}")(self.n, self.S, self.k, self._ptr(self.node_slot),
                                                   self._ptr(self.chain_of), self._ptr(self.N), self._ptr(self.u_ptr),
                                                   self.n_ulevels, self._ptr(self.u_nodes), self._ptr(g), self._ptr(f),
                                                   self._ptr(P))
        return f

    def mobius(self, g):
        g, suf, dt = self._prep(g)
        f = np.empty(self.n, dt)
        P = np.empty(self.S, dt)
        getattr(_load(), f"mzcpu_mobius_{suf}")(self.S, self.k, self._ptr(self.node_slot), self._ptr(self.chain_of),
                                                 self._ptr(self.N), self._ptr(self.lvl_ptr), self.nlevels,
                                                 self._ptr(self.lvl_nodes), self._ptr(g), self._ptr(f), self._ptr(P))
        return f
