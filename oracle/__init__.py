"""CPU oracle for the zeta and Moebius transforms on a finite poset.

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package. The GPU
library and its Python binding never import it, and it shares no code with
them: it computes everything from the definitions below, slowly and plainly,
in exact arithmetic.

What each function follows (arxiv 2211.13706, Pegolotti, Seifert, Pueschel):

* ``topological_order``  - Sec. 2.1: a list in which x < y puts x after y
  (first element a largest one). Kahn's algorithm; a cycle raises.
* ``closure``            - Sec. 2.1 / Cor. 1: x <= y iff there is a path from
  y to x; Z[x, y] = 1 iff y <= x. Built from out(x) = {x} union the out-sets
  of the children of x, bottom-up.
* ``zeta``               - Thm. 1 / Cor. 1, left: g(x) = sum_{y <= x} f(y).
* ``mobius_function``    - Thm. 1: the recursive mu (C helper ``mu.c``).
* ``mobius``             - Thm. 1 / Cor. 1, right: f(x) = sum_{y <= x} mu(y,x) g(y)
  (``method="mu"``), or the triangular solve Z f = g by back-substitution,
  which Sec. 2.2 names as the direct way (``method="backsub"``).
* ``zeta_T`` / ``mobius_T`` - the transposed matrices Z^T and M^T (up-set sums),
  defined here as plain matrix transposes; the paper has no adjoint section.
* ``niv``                - Sec. 2.4: niv_j(x) = the largest element of
  out(x) intersected with chain Z_j, or infinity.
* ``heights``            - Sec. 4, antichain decomposition (Alg. 6): level 1
  holds the minimal elements, every other x sits one above its highest child.
* ``reach`` / ``zeta_rows`` / ``mobius_residual_rows`` - the same definitions
  for single rows of very large posets, with out(x) found by breadth-first
  search (scipy), for sampled checks where O(n^2) is out of reach.

Exactness. Integer inputs are summed in Python integers. Floating-point
inputs are converted exactly to integers times a power of two, summed exactly,
and rounded once (Python's int / int division rounds correctly), so every
float result is the exact result correctly rounded to fp64. A ``F32C`` value
is the exact sum hi + lo of its two fp32 planes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

__all__ = ["CycleError", "topological_order", "closure", "zeta", "zeta_T", "mobius_function",
           "mobius", "mobius_T", "niv", "heights", "reach", "zeta_rows", "mobius_residual_rows",
           "exact_values", "load_library"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


class CycleError(ValueError):
    pass


def load_library():
    """Compile (if needed) and load the C helper of the oracle."""
    global _LIB
    if _LIB is not None:
        return _LIB
    out_dir = os.path.join(_HERE, "_build")
    so = os.path.join(out_dir, "libmzoracle.so")
    src = os.path.join(_HERE, "mu.c")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        os.makedirs(out_dir, exist_ok=True)
        tmp = so + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", tmp])
        os.replace(tmp, so)
    lib = ctypes.CDLL(so)
    lib.orc_mobius_function.restype = ctypes.c_int
    lib.orc_mobius_function.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    _LIB = lib
    return lib


# ----------------------------------------------------------------------------- structure

def _children(n, src, dst):
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    kids = [[] for _ in range(n)]
    for u, v in zip(src.tolist(), dst.tolist()):
        kids[u].append(v)
    return kids


def topological_order(n, src, dst) -> np.ndarray:
    """Kahn's algorithm from the sources: order[0] is a largest element."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("node id out of range")
    indeg = np.bincount(dst, minlength=n).astype(np.int64)
    kids = _children(n, src, dst)
    stack = [x for x in range(n) if indeg[x] == 0]
    order = []
    while stack:
        x = stack.pop()
        order.append(x)
        for v in kids[x]:
            indeg[v] -= 1
            if indeg[v] == 0:
                stack.append(v)
    if len(order) != n:
        raise CycleError("graph has a cycle")
    return np.array(order, dtype=np.int64)


def closure(n, src, dst) -> np.ndarray:
    """Zeta matrix Z (bool n x n): Z[x, y] = True iff y <= x (path from x to y, or y == x)."""
    order = topological_order(n, src, dst)
    kids = _children(n, src, dst)
    Z = np.zeros((n, n), dtype=bool)
    for x in order[::-1].tolist():          # bottom-up: children first
        Z[x, x] = True
        for v in kids[x]:
            Z[x] |= Z[v]
    return Z


def heights(n, src, dst) -> np.ndarray:
    """Level of every element: 1 for minimal elements, else 1 + the highest child level."""
    order = topological_order(n, src, dst)
    kids = _children(n, src, dst)
    h = np.zeros(n, dtype=np.int64)
    for x in order[::-1].tolist():
        h[x] = 1 + max((h[v] for v in kids[x]), default=0)
    return h


def niv(Z: np.ndarray, chain_id: np.ndarray) -> np.ndarray:
    """niv matrix: N[x, j] = niv_j(x) (an element id) or -1 for infinity.

    niv_j(x) is the element z of out(x) on chain j with every other element of
    out(x) on chain j below it. Raises if chain j is not totally ordered there."""
    n = Z.shape[0]
    chain_id = np.asarray(chain_id)
    k = int(chain_id.max()) + 1 if n else 0
    N = np.full((n, k), -1, dtype=np.int64)
    for x in range(n):
        for j in range(k):
            cand = np.flatnonzero(Z[x] & (chain_id == j))
            if cand.size == 0:
                continue
            tops = [z for z in cand.tolist() if Z[z, cand].all()]
            if len(tops) != 1:
                raise ValueError(f"chain {j} is not totally ordered below element {x}")
            N[x, j] = tops[0]
    return N


# ----------------------------------------------------------------------------- exact values

def exact_values(a) -> tuple[list, int]:
    """Exact integers V and a scale s with a[i] == V[i] / 2**s.

    ``a`` is an int64 array, a float array, or a tuple (hi, lo) of fp32 arrays
    standing for hi + lo."""
    if isinstance(a, tuple):
        (Vh, sh), (Vl, sl) = (exact_values(np.ravel(np.asarray(t, dtype=np.float64))) for t in a)
        s = max(sh, sl)
        return [h << (s - sh) for h in Vh] if not Vl else \
            [(h << (s - sh)) + (l << (s - sl)) for h, l in zip(Vh, Vl)], s
    a = np.ravel(np.asarray(a))
    if np.issubdtype(a.dtype, np.integer):
        return [int(v) for v in a.tolist()], 0
    a = a.astype(np.float64)            # exact for fp32 and fp64
    if not np.all(np.isfinite(a)):
        raise ValueError("oracle takes finite values only")
    # a = m * 2**e with 0.5 <= |m| < 1, so a = M * 2**(e - 53) with M = m * 2**53 an exact integer
    m, e = np.frexp(a)
    M = (m * float(1 << 53)).astype(np.int64)
    t = e.astype(np.int64) - 53
    nz = M != 0
    s = int(max(0, -int(t[nz].min()))) if nz.any() else 0
    return [int(Mi) << int(ti + s) if Mi else 0 for Mi, ti in zip(M.tolist(), t.tolist())], s


def _round(V: list, s: int, like) -> np.ndarray:
    """Exact V / 2**s: integers for integer inputs, else correctly rounded fp64."""
    if s == 0 and not _is_float(like):
        out = np.array(V, dtype=object)
        if any(abs(v) >= (1 << 63) for v in V):
            raise OverflowError("result does not fit int64")
        return out.astype(np.int64)
    den = 1 << s
    return np.array([v / den for v in V], dtype=np.float64)


def _is_float(like) -> bool:
    return isinstance(like, tuple) or np.issubdtype(np.asarray(like).dtype, np.floating)


def _columns(a):
    """Split a [n] or [n][B] input (or an (hi, lo) tuple of them) into columns."""
    if isinstance(a, tuple):
        hi, lo = (np.asarray(t) for t in a)
        if hi.ndim == 1:
            return [(hi, lo)], False
        return [(hi[:, b], lo[:, b]) for b in range(hi.shape[1])], True
    a = np.asarray(a)
    if a.ndim == 1:
        return [a], False
    return [a[:, b] for b in range(a.shape[1])], True


def _stack(cols, batched):
    return np.stack(cols, axis=1) if batched else cols[0]


# ----------------------------------------------------------------------------- transforms

def _apply_01(W: np.ndarray, a) -> np.ndarray:
    """Exact W @ a for a 0/1 (or small integer) matrix W."""
    cols, batched = _columns(a)
    res = []
    for col in cols:
        V, s = exact_values(col)
        Vo = np.array(V, dtype=object)
        out = []
        for x in range(W.shape[0]):
            nz = np.flatnonzero(W[x])
            if W.dtype == bool:
                out.append(int(sum(Vo[nz].tolist())))
            else:
                out.append(int(sum(int(w) * v for w, v in zip(W[x, nz].tolist(), Vo[nz].tolist()))))
        res.append(_round(out, s, col))
    return _stack(res, batched)


def zeta(Z: np.ndarray, f) -> np.ndarray:
    """g(x) = sum_{y <= x} f(y) (Thm. 1 left; g = Z f, Cor. 1)."""
    return _apply_01(Z, f)


def zeta_T(Z: np.ndarray, h) -> np.ndarray:
    """r(y) = sum_{x : y <= x} h(x) (r = Z^T h: sums over up-sets)."""
    return _apply_01(np.ascontiguousarray(Z.T), h)


def mobius_function(Z: np.ndarray, order: np.ndarray | None = None) -> np.ndarray:
    """mu[y, x] = mu(y, x) by Thm. 1's recursion (C helper, overflow-checked int64)."""
    n = Z.shape[0]
    if order is None:
        # any linear extension: sort by the number of elements below (a strict
        # superset of a down-set is strictly larger), largest first
        order = np.argsort(-Z.sum(axis=1), kind="stable")
    Zb = np.ascontiguousarray(Z, dtype=np.uint8)
    order = np.ascontiguousarray(order, dtype=np.int64)
    mu = np.zeros((n, n), dtype=np.int64)
    rc = load_library().orc_mobius_function(n, Zb.ctypes.data, order.ctypes.data, mu.ctypes.data)
    if rc != 0:
        raise OverflowError("mobius function overflowed int64")
    return mu


def mobius(Z: np.ndarray, g, method: str = "mu", mu: np.ndarray | None = None) -> np.ndarray:
    """f(x) = sum_{y <= x} mu(y, x) g(y) (Thm. 1 right; f = M g with M[x, y] = mu(y, x)).

    ``method="backsub"`` solves Z f = g instead, bottom-up:
    f(x) = g(x) - sum_{y < x} f(y), in exact arithmetic."""
    if method == "mu":
        if mu is None:
            mu = mobius_function(Z)
        return _apply_01(np.ascontiguousarray(mu.T), g)
    if method != "backsub":
        raise ValueError(method)
    n = Z.shape[0]
    order = np.argsort(Z.sum(axis=1), kind="stable")    # fewest elements below first
    cols, batched = _columns(g)
    res = []
    for col in cols:
        G, s = exact_values(col)
        F = [None] * n
        for x in order.tolist():
            below = np.flatnonzero(Z[x])
            acc = G[x]
            for y in below.tolist():
                if y != x:
                    acc -= F[y]
            F[x] = acc
        res.append(_round(F, s, col))
    return _stack(res, batched)


def mobius_T(Z: np.ndarray, h, mu: np.ndarray | None = None) -> np.ndarray:
    """r = M^T h: r(y) = sum_{x : y <= x} mu(y, x) h(x)."""
    if mu is None:
        mu = mobius_function(Z)
    return _apply_01(mu, h)


# ----------------------------------------------------------------------------- large posets: single rows

def _csr(n, src, dst):
    import scipy.sparse as sp
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    return sp.csr_matrix((np.ones(src.size, dtype=np.int8), (src, dst)), shape=(n, n))


def reach(n, src, dst, x: int, csr=None) -> np.ndarray:
    """out(x): every element reachable from x, x included (breadth-first search)."""
    from scipy.sparse.csgraph import breadth_first_order
    if csr is None:
        csr = _csr(n, src, dst)
    return np.sort(breadth_first_order(csr, int(x), directed=True, return_predecessors=False))


def zeta_rows(n, src, dst, f, rows) -> np.ndarray:
    """g(x) = sum_{y in out(x)} f(y) for the listed x only (exact, then rounded as in ``zeta``)."""
    csr = _csr(n, src, dst)
    cols, batched = _columns(f)
    res = []
    for col in cols:
        out = []
        for x in rows:
            r = reach(n, src, dst, x, csr)
            if isinstance(col, tuple):
                part = (col[0][r], col[1][r])
            else:
                part = col[r]
            V, s = exact_values(part)
            out.append(_round([sum(V)], s, col)[0])
        res.append(np.array(out))
    return _stack(res, batched)


def mobius_residual_rows(n, src, dst, f_out, g, rows):
    """For each listed x: (sum_{y in out(x)} f_out(y) - g(x), sum_{y in out(x)} |f_out(y)| + |g(x)|).

    A Moebius result f_out is correct iff Z f_out = g (Cor. 1), so the
    residual is zero for exact results; the second value is the magnitude the
    residual is measured against. Both are exact, then rounded to fp64 (or
    kept as integers for integer inputs)."""
    csr = _csr(n, src, dst)
    fc, batched = _columns(f_out)
    gc, _ = _columns(g)
    res, mag = [], []
    for col_f, col_g in zip(fc, gc):
        r_out, m_out = [], []
        for x in rows:
            r = reach(n, src, dst, x, csr)
            part = (col_f[0][r], col_f[1][r]) if isinstance(col_f, tuple) else col_f[r]
            gx = (col_g[0][x:x + 1], col_g[1][x:x + 1]) if isinstance(col_g, tuple) else col_g[x:x + 1]
            Vf, sf = exact_values(part)
            Vg, sg = exact_values(gx)
            s = max(sf, sg)
            tot = sum(v << (s - sf) for v in Vf) - (Vg[0] << (s - sg))
            absv = sum(abs(v) << (s - sf) for v in Vf) + (abs(Vg[0]) << (s - sg))
            if _is_float(col_f) or _is_float(col_g):
                r_out.append(tot / (1 << s))
                m_out.append(absv / (1 << s))
            else:
                r_out.append(tot)
                m_out.append(absv)
        res.append(np.array(r_out))
        mag.append(np.array(m_out))
    return _stack(res, batched), _stack(mag, batched)

