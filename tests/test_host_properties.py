"""Property tests of the host build on random small DAGs (hypothesis; host only):
the chains of Alg. 1 are a minimum path cover (k = n - maximum matching, the matching
computed by networkx), every chain is a path of edges, the niv map equals the oracle's,
the heights equal the oracle's, and the sparse and dense maps agree."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
nx = pytest.importorskip("networkx")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
import paper_2211_13706_gb300 as mz  # noqa: E402


@st.composite
def dags(draw):
    n = draw(st.integers(1, 24))
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    chosen = draw(st.lists(st.sampled_from(pairs), max_size=60)) if pairs else []
    perm = draw(st.permutations(range(n)))          # hide the order in the ids
    src = np.array([perm[i] for i, _ in chosen], np.int32)
    dst = np.array([perm[j] for _, j in chosen], np.int32)
    return n, src, dst


@settings(max_examples=150, deadline=None)
@given(dags())
def test_path_cover_niv_and_heights(g):
    n, src, dst = g
    plan = mz.Plan(n, src, dst, None, host_only=True, niv_format=1)
    info = plan.info
    # k = n - |maximum matching| of the split graph (Alg. 1)
    B = nx.Graph()
    B.add_nodes_from((("u", x) for x in range(n)))
    B.add_nodes_from((("v", x) for x in range(n)))
    B.add_edges_from((("u", int(a)), ("v", int(b))) for a, b in zip(src, dst))
    top = [("u", x) for x in range(n)]
    M = nx.bipartite.maximum_matching(B, top_nodes=top)
    assert info["k"] == n - len(M) // 2
    # each chain is a path of edges, bottom to top
    cid, cpos = plan.export(mz.MZ_EXPORT_CHAIN_ID), plan.export(mz.MZ_EXPORT_CHAIN_POS)
    edges = set(zip(src.tolist(), dst.tolist()))
    for c in range(info["k"]):
        members = sorted(np.flatnonzero(cid == c).tolist(), key=lambda x: cpos[x])
        for lo, hi in zip(members, members[1:]):
            assert (hi, lo) in edges
    Z = oracle.closure(n, src, dst)
    assert np.array_equal(plan.export(mz.MZ_EXPORT_NIV), oracle.niv(Z, cid))
    assert np.array_equal(plan.export(mz.MZ_EXPORT_LEVEL), oracle.heights(n, src, dst))
    sparse = mz.Plan(n, src, dst, None, host_only=True, niv_format=2)
    assert np.array_equal(sparse.export(mz.MZ_EXPORT_NIV), plan.export(mz.MZ_EXPORT_NIV))
    assert np.array_equal(sparse.export(mz.MZ_EXPORT_ULEVEL), plan.export(mz.MZ_EXPORT_ULEVEL))
