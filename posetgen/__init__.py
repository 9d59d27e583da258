"""Seeded synthetic posets and poset functions.

This module only draws random inputs. It holds none of the transform
arithmetic, so both the independent CPU oracle and the GPU path can consume
the same instances without sharing any method code.

Conventions (the paper's, Sec. 2.1): a DAG edge ``u -> v`` means ``v <= u``
(v is a successor of u). A *rank* is a topological index: rank 0 is a largest
element, so every edge goes from a lower rank to a higher rank.

Workload recipe (planted chains plus cross-chain edges), used for every
synthetic instance in the tests and the benchmark:

* ``rank`` is a uniform random permutation of the n node ids.
* The nodes are split into ``k`` chains of balanced sizes (``n // k`` or
  ``n // k + 1``) by a uniform random assignment. Inside a chain the members
  are linked in rank order by an edge from each member to the next one, so
  every chain is totally ordered.
* Cross-chain edges go from a node to a node of higher rank on another chain,
  so the graph is acyclic by construction. Two recipes:
    - ``cross_p``: every such ordered pair independently with probability p;
    - ``cross_deg``: each node draws a Poisson(d) number of targets, uniform
      among the higher-rank nodes of other chains (duplicates removed).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = ["Poset", "planted_chain_poset", "planted_batch_specs", "random_dag_tiny", "er_dag", "boolean_lattice",
           "divisor_lattice", "chain_poset", "antichain_poset", "paper_example",
           "function_values", "sub_poset"]


@dataclass
class Poset:
    """A DAG on nodes 0..n-1. ``src[i] -> dst[i]`` means ``dst[i] <= src[i]``."""

    n: int
    src: np.ndarray          # int32 [m]
    dst: np.ndarray          # int32 [m]
    chain_id: np.ndarray | None = None   # int32 [n] planted chain partition (optional)
    rank: np.ndarray | None = None       # int64 [n] a topological index (optional)
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    @property
    def k(self) -> int | None:
        return None if self.chain_id is None else int(self.chain_id.max()) + 1 if self.n else 0


def _balanced_chains(rng, n, k):
    """Random balanced assignment of n nodes to k chains."""
    perm = rng.permutation(n)
    chain_id = np.empty(n, dtype=np.int32)
    chain_id[perm] = np.arange(n, dtype=np.int64) % k
    return chain_id


def planted_chain_poset(n: int, k: int, seed: int, *, cross_p: float | None = None,
                        cross_deg: float | None = None) -> Poset:
    """Planted-chain random poset (recipe in the module docstring)."""
    if n < 1 or k < 1 or k > n:
        raise ValueError("need 1 <= k <= n")
    rng = np.random.default_rng(seed)
    rank = rng.permutation(n).astype(np.int64)          # rank[node]
    node_at_rank = np.empty(n, dtype=np.int64)
    node_at_rank[rank] = np.arange(n)
    chain_id = _balanced_chains(rng, n, k)

    # chain edges: members of each chain in rank order, consecutive pairs
    order = np.lexsort((rank, chain_id))                 # by chain, then rank
    same = chain_id[order[:-1]] == chain_id[order[1:]]
    c_src = order[:-1][same]
    c_dst = order[1:][same]

    if cross_p is not None:
        # every ordered pair (rank u < rank v, other chain) independently w.p. p
        iu, iv = np.triu_indices(n, k=1)                 # indices into rank order
        keep = rng.random(iu.shape[0]) < cross_p
        u = node_at_rank[iu[keep]]
        v = node_at_rank[iv[keep]]
        ok = chain_id[u] != chain_id[v]
        x_src, x_dst = u[ok], v[ok]
    elif cross_deg is not None:
        cnt = rng.poisson(cross_deg, size=n)
        u = np.repeat(np.arange(n, dtype=np.int64), cnt)
        ru = rank[u]
        room = (n - 1) - ru                              # number of higher-rank nodes
        has = room > 0
        u, ru, room = u[has], ru[has], room[has]
        tgt = np.full(u.shape[0], -1, dtype=np.int64)
        pending = np.arange(u.shape[0])
        for _ in range(8):                               # rejection rounds for same-chain draws
            if pending.size == 0:
                break
            r = ru[pending] + 1 + (rng.random(pending.size) * room[pending]).astype(np.int64)
            r = np.minimum(r, n - 1)
            v = node_at_rank[r]
            good = chain_id[v] != chain_id[u[pending]]
            tgt[pending[good]] = v[good]
            pending = pending[~good]
        ok = tgt >= 0
        x_src, x_dst = u[ok], tgt[ok]
        key = np.sort(x_src * n + x_dst)                  # sorted unique (same result as np.unique)
        key = key[np.concatenate([[True], key[1:] != key[:-1]])] if key.size else key
        x_src, x_dst = key // n, key % n
    else:
        x_src = x_dst = np.zeros(0, dtype=np.int64)

    src = np.concatenate([c_src, x_src]).astype(np.int32)
    dst = np.concatenate([c_dst, x_dst]).astype(np.int32)
    return Poset(n=n, src=src, dst=dst, chain_id=chain_id, rank=rank,
                 name=f"planted(n={n},k={k},seed={seed})")


def planted_batch_specs(count: int, seed: int, n_range=(1024, 65536), k_range=(4, 256)):
    """(n, k, seed) of `count` planted posets for a batch workload: n and k log-uniform
    in their ranges (rounded; k at most n // 2), one seed per poset."""
    rng = np.random.default_rng(seed)
    n = np.rint(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1]), count))).astype(np.int64)
    k = np.rint(np.exp(rng.uniform(np.log(k_range[0]), np.log(k_range[1]), count))).astype(np.int64)
    k = np.maximum(1, np.minimum(k, n // 2))
    seeds = rng.integers(0, 2 ** 31 - 1, count)
    return [(int(a), int(b), int(c)) for a, b, c in zip(n, k, seeds)]


def random_dag_tiny(n: int, p: float, seed: int) -> Poset:
    """Erdos-Renyi DAG: each pair (i, j), i < j in a random order, is an edge w.p. p."""
    rng = np.random.default_rng(seed)
    rank = rng.permutation(n).astype(np.int64)
    node_at_rank = np.empty(n, dtype=np.int64)
    node_at_rank[rank] = np.arange(n)
    iu, iv = np.triu_indices(n, k=1)
    keep = rng.random(iu.shape[0]) < p
    src = node_at_rank[iu[keep]].astype(np.int32)
    dst = node_at_rank[iv[keep]].astype(np.int32)
    return Poset(n=n, src=src, dst=dst, rank=rank, name=f"er(n={n},p={p},seed={seed})")


def er_dag(n: int, degree: float, seed: int) -> Poset:
    """The paper's random DAGs (Sec. 5): Erdos-Renyi on a random order, an ordered pair
    (earlier, later) is an edge with probability degree / (n - 1), so the average total
    degree is `degree`. Sampled as the binomial number of edges drawn uniformly (pairs
    drawn twice are merged)."""
    rng = np.random.default_rng(seed)
    m = int(rng.binomial(n * (n - 1) // 2, min(1.0, degree / max(1, n - 1))))
    a = rng.integers(0, n, size=2 * m + 16)
    b = rng.integers(0, n, size=2 * m + 16)
    keep = a < b
    a, b = a[keep][:m], b[keep][:m]
    key = np.sort(a.astype(np.int64) * n + b)
    key = key[np.concatenate([[True], key[1:] != key[:-1]])] if key.size else key
    a, b = key // n, key % n
    perm = rng.permutation(n)                              # node ids in a random order
    return Poset(n=n, src=perm[a].astype(np.int32), dst=perm[b].astype(np.int32),
                 name=f"er(n={n},deg={degree},seed={seed})")


def boolean_lattice(m: int) -> Poset:
    """Subsets of {0..m-1} ordered by inclusion; node id = bitmask. Cover edges S -> S minus one element."""
    n = 1 << m
    s = np.arange(n, dtype=np.int64)
    src, dst = [], []
    for b in range(m):
        has = (s >> b) & 1 == 1
        src.append(s[has])
        dst.append(s[has] ^ (1 << b))
    return Poset(n=n, src=np.concatenate(src).astype(np.int32),
                 dst=np.concatenate(dst).astype(np.int32), name=f"boolean({m})")


def divisor_lattice(N: int) -> tuple[Poset, np.ndarray]:
    """Divisors of N ordered by divisibility. Cover edges d -> d/p for primes p | d.

    Returns the poset and the divisor value of each node id (ascending)."""
    divs = np.array([d for d in range(1, N + 1) if N % d == 0], dtype=np.int64)
    index = {int(d): i for i, d in enumerate(divs)}
    primes = [p for p in range(2, N + 1) if N % p == 0 and all(p % q for q in range(2, int(p ** 0.5) + 1))]
    src, dst = [], []
    for d in divs:
        for p in primes:
            if d % p == 0:
                src.append(index[int(d)])
                dst.append(index[int(d // p)])
    return (Poset(n=len(divs), src=np.array(src, dtype=np.int32), dst=np.array(dst, dtype=np.int32),
                  name=f"divisors({N})"), divs)


def chain_poset(n: int, seed: int = 0) -> Poset:
    """A total order on n nodes in a random id order: top -> ... -> bottom."""
    rng = np.random.default_rng(seed)
    order = rng.permutation(n)
    return Poset(n=n, src=order[:-1].astype(np.int32), dst=order[1:].astype(np.int32),
                 chain_id=np.zeros(n, dtype=np.int32), name=f"chain({n})")


def antichain_poset(n: int) -> Poset:
    """n pairwise incomparable nodes (no edges)."""
    return Poset(n=n, src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32),
                 chain_id=np.arange(n, dtype=np.int32), name=f"antichain({n})")


def paper_example() -> Poset:
    """The 12-element cover graph of the paper's running example (Sec. 2.2, matrix A).

    Node id i-1 stands for the paper's element x_i. Edges are the 1-entries of A
    (row = source, column = target); they are read from the text fixture
    tests/golden/paper_example_A.txt by the tests, and repeated here so the
    benchmark and smoke test need no file access."""
    rows = {
        1: [3, 4, 6], 2: [4, 5], 3: [7, 8], 4: [7, 9], 5: [10], 6: [8, 9],
        7: [10], 8: [11], 9: [12], 10: [11, 12],
    }
    src = [a - 1 for a, bs in rows.items() for _ in bs]
    dst = [b - 1 for bs in rows.values() for b in bs]
    return Poset(n=12, src=np.array(src, np.int32), dst=np.array(dst, np.int32), name="paper_example")


def sub_poset(p: Poset, keep: np.ndarray) -> tuple[Poset, np.ndarray]:
    """Induced sub-DAG on the nodes where ``keep`` is True (renumbered in id order).

    Only edges with both ends kept survive, so the result is the induced
    poset only when the kept set is convex (e.g. a down-set or an up-set)."""
    keep = np.asarray(keep, dtype=bool)
    new_id = np.full(p.n, -1, dtype=np.int64)
    old = np.flatnonzero(keep)
    new_id[old] = np.arange(old.size)
    e = keep[p.src] & keep[p.dst]
    chain = None
    if p.chain_id is not None:
        _, chain = np.unique(p.chain_id[old], return_inverse=True)
        chain = chain.astype(np.int32)
    return (Poset(n=int(old.size), src=new_id[p.src[e]].astype(np.int32),
                  dst=new_id[p.dst[e]].astype(np.int32), chain_id=chain,
                  name=p.name + "[sub]"), old)


def function_values(n: int, batch: int, kind: str, seed: int) -> np.ndarray:
    """Poset function values, layout [n][batch] (node-major, batch contiguous).

    kinds: ``i64:A`` uniform integers in [-A, A]; ``f64u`` uniform [-1, 1];
    ``f32u`` the same rounded to fp32; ``f64ln`` / ``f32ln`` sign * exp(3 N(0,1))
    (log-normal, sigma = 3, random signs)."""
    rng = np.random.default_rng(seed)
    shape = (n, batch)
    if kind.startswith("i64:"):
        a = int(kind.split(":")[1])
        return rng.integers(-a, a + 1, size=shape, dtype=np.int64)
    if kind in ("f64u", "f32u"):
        x = rng.uniform(-1.0, 1.0, size=shape)
    elif kind in ("f64ln", "f32ln"):
        x = np.exp(3.0 * rng.standard_normal(shape)) * rng.choice([-1.0, 1.0], size=shape)
    else:
        raise ValueError(kind)
    return x.astype(np.float32) if kind.startswith("f32") else x
